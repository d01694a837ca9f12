// Serving loop: continuous batching of solve requests on one GPU.
//
// Requests (a medium, a decomposition, nrhs sources, GMRES options) arrive at
// any time through hd_submit.  A request is admitted into a slot as soon as a
// slot is free and its device memory (context tables, factors, Krylov bases,
// staging, vectors) fits in what is left of the HBM budget; admitted requests
// run at the same time, each on its own stream and worker thread, so their
// kernels overlap on the device, and a request that arrives while others run
// starts as soon as a slot and memory free up.  Every request keeps its
// factors and Krylov basis resident for its whole lifetime.  Device memory
// comes from the stream-ordered allocator, so no allocation or free
// synchronises the device and stalls other slots.  The kernels are
// deterministic and requests share no device data, so a result is the same
// alone and in the mix.  A request whose nrhs right-hand sides would not fit
// the budget at once is solved in sub-batches that do.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hd_internal.cuh"

namespace hd {

using clk = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  hd_grid grid;
  int nbx = 1, nby = 1, overlap = 0, own = 1;
  std::vector<int32_t> cut_x, cut_y;
  int precision = HD_C64;
  int nrhs = 1;
  hd_gmres_opts opts;
  const double *c_host = nullptr;
  const void *f_host = nullptr;
  void *x_host = nullptr;
  size_t bytes = 0;      // device bytes reserved while running
  int batch = 1;         // right-hand sides per lockstep solve
  int status = HD_PENDING;
  std::string error;
  std::vector<hd_gmres_stats> stats;
  clk::time_point t_submit, t_start, t_done;
};

}  // namespace hd

struct hd_server {
  size_t budget = 0, in_use = 0, peak_in_use = 0;
  int max_slots = 1, device = 0, running = 0, peak_running = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<hd::Request>> queue;
  std::map<uint64_t, std::shared_ptr<hd::Request>> live;   // submitted, not yet collected
  std::vector<std::thread> workers;
  uint64_t completed = 0;
  // the requests' device memory: a pool of the server's own that keeps up to the budget
  // mapped between requests (a release threshold of zero would hand it back to the
  // driver at every synchronisation and map it again for the next request)
  cudaMemPool_t pool = nullptr;
};

namespace hd {

// Box extents along one axis (same rule as the context set-up, Sec. 2).
static bool axis_extents(int n_in, int npml, int nb, int overlap, const std::vector<int32_t> &cut,
                         std::vector<int> &ext) {
  std::vector<int32_t> c(nb + 1);
  for (int i = 0; i <= nb; ++i) c[i] = cut.empty() ? npml + (int32_t)(((int64_t)i * n_in) / nb) : cut[i];
  ext.resize(nb);
  for (int i = 0; i < nb; ++i) {
    int e0 = c[i] - npml - (i > 0 ? overlap : 0);
    int e1 = c[i + 1] + npml + (i < nb - 1 ? overlap : 0);
    if (e1 <= e0) return false;
    ext[i] = e1 - e0;
  }
  return true;
}

// Device bytes a request holds while it runs with `batch` right-hand sides per solve.
static size_t request_bytes(const Request &q, int batch) {
  std::vector<int> ex, ey;
  if (!axis_extents(q.grid.nx, q.grid.npml, q.nbx, q.overlap, q.cut_x, ex) ||
      !axis_extents(q.grid.ny, q.grid.npml, q.nby, q.overlap, q.cut_y, ey))
    return (size_t)-1;
  const size_t cs = compute_bytes(q.precision & 0xff);
  const bool sym = (q.precision & HD_SYMMETRIC) != 0;
  size_t factor = 0, staging = 0, work = 0;
  for (int a : ey)
    for (int b : ex) {
      const size_t mt = (b + 15) / 16;
      const size_t mp8 = (b + 7) & ~7;
      factor += sym ? (size_t)a * mt * (mt + 1) / 2 * 256
                    : ((q.precision & HD_TCORE) ? ((q.precision & HD_TF32X3) ? 2 : 1) * (size_t)a * mp8 * mp8
                                                : (size_t)a * b * ((b + 3) & ~3));
      staging += (size_t)a * b;
      work += 2 * (size_t)b * b;
    }
  const size_t n = (size_t)(q.grid.nx + 2 * q.grid.npml) * (q.grid.ny + 2 * q.grid.npml);
  const size_t tables = 2 * n * 8 + ((size_t)1 << 20);   // k^2, centre coefficients, PML tables
  const size_t vecs = n * 8 + 2 * n * 16 * (size_t)batch;     // velocity, right-hand sides, solutions
  return store_bytes(q.precision & 0xff) * factor + cs * std::max(staging * batch, work) + krylov_bytes((int64_t)n, q.opts.restart, batch) +
         tables + vecs;
}

static void run_request(hd_server *srv, Request &q, cudaStream_t st) {
  const int64_t n = (int64_t)(q.grid.nx + 2 * q.grid.npml) * (q.grid.ny + 2 * q.grid.npml);
  const int B = q.batch;
  void *c_d = nullptr, *f_d = nullptr, *x_d = nullptr, *fac = nullptr, *kws = nullptr, *scr = nullptr;
  hd_ctx *ctx = nullptr;
  size_t fb = 0, kb = 0, sb = 0;
  auto fail = [&](int rc, const std::string &what) {
    q.status = rc;
    q.error = what + ": " + hd_last_error();
  };
  q.stats.assign(q.nrhs, hd_gmres_stats{});
  auto dalloc = [&](void **p, size_t bytes) {
    return srv->pool ? cudaMallocFromPoolAsync(p, bytes, srv->pool, st) : cudaMallocAsync(p, bytes, st);
  };
  do {
    if (dalloc(&c_d, sizeof(double) * n) != cudaSuccess || dalloc(&f_d, sizeof(double2) * n * B) != cudaSuccess ||
        dalloc(&x_d, sizeof(double2) * n * B) != cudaSuccess) {
      fail(HD_ERR_OOM, "device vectors");
      break;
    }
    if (cudaMemcpyAsync(c_d, q.c_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      fail(HD_ERR_CUDA, "velocity copy");
      break;
    }
    hd_decomp dec{q.nbx, q.nby, q.overlap, q.cut_x.empty() ? nullptr : q.cut_x.data(),
                  q.cut_y.empty() ? nullptr : q.cut_y.data(), q.own};
    int rc = hd_setup_medium(&ctx, &q.grid, &dec, reinterpret_cast<const double *>(c_d), q.precision, st);
    if (rc) { fail(rc, "hd_setup_medium"); break; }
    hd_query_workspace(ctx, B, q.opts.restart, &fb, &kb, &sb);
    if (dalloc(&fac, fb) != cudaSuccess || dalloc(&kws, kb) != cudaSuccess || dalloc(&scr, sb) != cudaSuccess) {
      fail(HD_ERR_OOM, "workspaces");
      break;
    }
    rc = hd_factor_subdomains(ctx, fac, fb, scr, sb, st);
    if (rc) { fail(rc, "hd_factor_subdomains"); break; }
    // the substitution's launch shape: tuned once per shape class in this process (the first
    // request of a class pays for the timing runs; f_d and x_d are free until the solve)
    if (!lookup_tuning(ctx) && hd_autotune(ctx, f_d, x_d, scr, sb, nullptr, nullptr, nullptr, st) != HD_OK)
      cudaGetLastError();
    int worst = HD_OK;
    for (int r0 = 0; r0 < q.nrhs; r0 += B) {
      const int g = std::min(B, q.nrhs - r0);
      const double2 *fh = reinterpret_cast<const double2 *>(q.f_host) + (int64_t)r0 * n;
      if (cudaMemcpyAsync(f_d, fh, sizeof(double2) * n * g, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        worst = HD_ERR_CUDA;
        break;
      }
      rc = hd_rhs_from_source(ctx, f_d, f_d, g, st);
      if (!rc) rc = hd_gmres_solve(ctx, f_d, x_d, g, &q.opts, kws, kb, scr, sb, q.stats.data() + r0, st);
      if (rc && rc != HD_ERR_NOT_CONVERGED) { worst = rc; break; }
      if (rc && !worst) worst = rc;
      double2 *xh = reinterpret_cast<double2 *>(q.x_host) + (int64_t)r0 * n;
      if (cudaMemcpyAsync(xh, x_d, sizeof(double2) * n * g, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        worst = HD_ERR_CUDA;
        break;
      }
    }
    q.status = worst;
    if (worst) q.error = hd_last_error();
  } while (false);
  if (ctx) hd_destroy(ctx);
  for (void *p : {c_d, f_d, x_d, fac, kws, scr})
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
}

static void worker_main(hd_server *srv) {
  cudaSetDevice(srv->device);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  for (;;) {
    std::shared_ptr<Request> q;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      // admit the oldest request once its memory fits (first come, first served)
      srv->cv_work.wait(lk, [&] {
        return srv->stopping || (!srv->queue.empty() && srv->in_use + srv->queue.front()->bytes <= srv->budget);
      });
      if (srv->stopping) break;   // admitted requests finish; queued ones are dropped
      q = srv->queue.front();
      srv->queue.pop_front();
      srv->in_use += q->bytes;
      srv->peak_in_use = std::max(srv->peak_in_use, srv->in_use);
      srv->running += 1;
      srv->peak_running = std::max(srv->peak_running, srv->running);
    }
    q->t_start = clk::now();
    run_request(srv, *q, st);
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      q->t_done = clk::now();
      srv->in_use -= q->bytes;
      srv->running -= 1;
      srv->completed += 1;
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace hd

using namespace hd;

extern "C" {

int hd_server_create(hd_server **out, size_t hbm_budget_bytes, int32_t max_slots, int32_t device) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) {
    set_error("hd_server_create: bad argument");
    return HD_ERR_INVALID;
  }
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    set_error("hd_server_create: no such CUDA device");
    return HD_ERR_INVALID;
  }
  hd_server *s = new hd_server();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->device = device;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&s->pool, &props) == cudaSuccess) {
    uint64_t keep = hbm_budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    s->pool = nullptr;   // fall back to the device's default pool
    cudaGetLastError();
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return HD_OK;
}

int hd_submit(hd_server *s, const hd_grid *grid, const hd_decomp *dec, const double *c_host, const void *f_host,
              int32_t nrhs, int32_t precision, const hd_gmres_opts *opts, void *x_host, uint64_t *ticket) {
  if (!s || !grid || !dec || !c_host || !f_host || !opts || !x_host || !ticket || nrhs < 1 || opts->restart < 1 ||
      opts->restart > HD_MAX_RESTART ||
      ((precision & 0xff) != HD_C64 && (precision & 0xff) != HD_C128 && (precision & 0xff) != HD_C64_H &&
       (precision & 0xff) != HD_C64_B) ||
      (precision & ~(0xff | HD_SYMMETRIC | HD_TCORE | HD_TF32X3 | HD_SMOOTH)) ||
      ((precision & HD_TF32X3) && !(precision & HD_TCORE)) ||
      ((precision & HD_TCORE) && ((precision & 0xff) != HD_C64 || (precision & HD_SYMMETRIC)))) {
    set_error("hd_submit: bad argument");
    return HD_ERR_INVALID;
  }
  auto q = std::make_shared<Request>();
  q->grid = *grid;
  q->nbx = dec->nbx; q->nby = dec->nby; q->overlap = dec->overlap; q->own = dec->own_global_pml ? 1 : 0;
  if (dec->nbx < 1 || dec->nby < 1) { set_error("hd_submit: bad decomposition"); return HD_ERR_INVALID; }
  if (dec->cut_x) q->cut_x.assign(dec->cut_x, dec->cut_x + dec->nbx + 1);
  if (dec->cut_y) q->cut_y.assign(dec->cut_y, dec->cut_y + dec->nby + 1);
  q->precision = precision;
  q->nrhs = nrhs;
  q->opts = *opts;
  q->c_host = c_host; q->f_host = f_host; q->x_host = x_host;
  // largest lockstep batch whose memory fits the whole budget
  int batch = nrhs;
  while (batch > 1 && request_bytes(*q, batch) > s->budget) batch = (batch + 1) / 2;
  q->batch = batch;
  q->bytes = request_bytes(*q, batch);
  if (q->bytes == (size_t)-1) { set_error("hd_submit: bad decomposition"); return HD_ERR_INVALID; }
  if (q->bytes > s->budget) { set_error("hd_submit: one right-hand side needs more than the HBM budget"); return HD_ERR_OOM; }
  q->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) { set_error("hd_submit: server is shutting down"); return HD_ERR_INVALID; }
    q->ticket = s->next_ticket++;
    s->queue.push_back(q);
    s->live[q->ticket] = q;
    *ticket = q->ticket;
  }
  s->cv_work.notify_all();
  return HD_OK;
}

int hd_poll(hd_server *s, uint64_t ticket, hd_gmres_stats *stats, hd_request_info *info, int64_t timeout_us) {
  if (!s) { set_error("hd_poll: NULL server"); return HD_ERR_INVALID; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) { set_error("hd_poll: unknown or already collected ticket"); return HD_ERR_INVALID; }
  std::shared_ptr<Request> q = it->second;
  auto done = [&] { return q->t_done != clk::time_point{}; };
  if (!done() && timeout_us != 0) {
    if (timeout_us < 0) s->cv_done.wait(lk, done);
    else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  }
  if (!done()) return HD_PENDING;
  s->live.erase(it);
  lk.unlock();
  if (stats) std::memcpy(stats, q->stats.data(), sizeof(hd_gmres_stats) * q->nrhs);
  if (info) {
    info->queue_s = std::chrono::duration<double>(q->t_start - q->t_submit).count();
    info->run_s = std::chrono::duration<double>(q->t_done - q->t_start).count();
    info->latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
    info->device_bytes = q->bytes;
    info->batch = q->batch;
  }
  if (q->status != HD_OK) set_error(q->error);
  return q->status;
}

int hd_server_info(hd_server *s, hd_server_counters *out) {
  if (!s || !out) { set_error("hd_server_info: bad argument"); return HD_ERR_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int32_t)s->queue.size();
  out->running = s->running;
  out->peak_running = s->peak_running;
  out->completed = s->completed;
  out->bytes_in_use = s->in_use;
  out->peak_bytes_in_use = s->peak_in_use;
  out->budget_bytes = s->budget;
  return HD_OK;
}

int hd_server_destroy(hd_server *s) {
  if (!s) return HD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();   // admitted requests finish; queued ones are dropped
  if (s->pool) cudaMemPoolDestroy(s->pool);   // every allocation was freed and synchronised by its worker
  delete s;
  return HD_OK;
}

}  // extern "C"
