// C ABI of libhd: argument checks, context set-up (decomposition tables of
// Sec. 2), workspace sizing, error reporting and kernel timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hd_internal.cuh"

namespace hd {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

cudaError_t allow_smem_ptr(const void *kernel, size_t bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const size_t limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  if (bytes > limit) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  return HD_ERR_CUDA;
}

static int invalid(const std::string &msg) {
  set_error(msg);
  return HD_ERR_INVALID;
}

// ---------------------------------------------------------------- timers
static cudaEvent_t get_event(hd_ctx *ctx) {
  if (ctx->ev_next < ctx->ev_pool.size()) return ctx->ev_pool[ctx->ev_next++];
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  ctx->ev_pool.push_back(e);
  ctx->ev_next = ctx->ev_pool.size();
  return e;
}

void tic(hd_ctx *ctx, int cls, cudaStream_t st) {
  if (!ctx->profiling) return;
  cudaEvent_t a = get_event(ctx);
  if (!a) return;
  cudaEventRecord(a, st);
  ctx->ev_pending.push_back({cls, {a, nullptr}});
}

void toc(hd_ctx *ctx, int cls, cudaStream_t st, int nkernels) {
  ctx->t_launch[cls] += nkernels;
  if (!ctx->profiling || ctx->ev_pending.empty()) return;
  auto &p = ctx->ev_pending.back();
  if (p.first != cls || p.second.second) return;
  cudaEvent_t b = get_event(ctx);
  if (!b) return;
  cudaEventRecord(b, st);
  p.second.second = b;
}

int collect_timers(hd_ctx *ctx) {
  for (auto &p : ctx->ev_pending) {
    if (!p.second.second) continue;
    cudaEventSynchronize(p.second.second);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      ctx->t_ms[p.first] += ms;
    }
  }
  ctx->ev_pending.clear();
  ctx->ev_next = 0;
  return HD_OK;
}


static void free_ctx(hd_ctx *c) {
  if (!c) return;
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.second.exec);
  if (c->gstream) {
    cudaStreamSynchronize(c->gstream);
    cudaStreamDestroy(c->gstream);
  }
  if (c->gevent) cudaEventDestroy(c->gevent);
  if (c->d_k2) cudaFreeAsync(c->d_k2, c->stream);
  if (c->d_cc) cudaFreeAsync(c->d_cc, c->stream);
  if (c->d_gax_c) cudaFreeAsync(c->d_gax_c, c->stream);
  if (c->d_giax_f) cudaFreeAsync(c->d_giax_f, c->stream);
  if (c->d_gay_c) cudaFreeAsync(c->d_gay_c, c->stream);
  if (c->d_giay_f) cudaFreeAsync(c->d_giay_f, c->stream);
  if (c->d_lpool) cudaFreeAsync(c->d_lpool, c->stream);
  if (c->d_subs) cudaFreeAsync(c->d_subs, c->stream);
  if (c->d_axx) cudaFreeAsync(c->d_axx, c->stream);
  if (c->d_axy) cudaFreeAsync(c->d_axy, c->stream);
  if (c->d_nearx) cudaFreeAsync(c->d_nearx, c->stream);
  if (c->d_neary) cudaFreeAsync(c->d_neary, c->stream);
  if (c->d_status) cudaFreeAsync(c->d_status, c->stream);
  if (c->d_fflag) cudaFreeAsync(c->d_fflag, c->stream);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

// Owned ranges and extents along one axis (Sec. 2: x_{i,0}, x_{i,1}).
static int axis_ranges(int n_in, int npml, int nb, int overlap, const int32_t *cut, int own_global_pml,
                       std::vector<AxisDev> &out, std::vector<int32_t> &near, const char *name) {
  const int n = n_in + 2 * npml;
  std::vector<int32_t> c(nb + 1);
  for (int i = 0; i <= nb; ++i) c[i] = cut ? cut[i] : npml + (int32_t)(((int64_t)i * n_in) / nb);
  if (c[0] != npml || c[nb] != npml + n_in)
    return invalid(std::string(name) + ": cut points must start at npml and end at npml + n");
  for (int i = 0; i < nb; ++i) {
    if (c[i + 1] <= c[i]) return invalid(std::string(name) + ": cut points must increase");
    if (nb > 1 && c[i + 1] - c[i] < overlap + npml)
      return invalid(std::string(name) + ": every owned width must be at least overlap + npml");
  }
  out.resize(nb);
  near.assign(n, 0);
  for (int i = 0; i < nb; ++i) {
    AxisDev a;
    a.o0 = c[i];
    a.o1 = c[i + 1];
    a.e0 = c[i] - npml - (i > 0 ? overlap : 0);
    a.e1 = c[i + 1] + npml + (i < nb - 1 ? overlap : 0);
    if (a.e0 < 0 || a.e1 > n) return invalid(std::string(name) + ": an overlapping box leaves the domain");
    if (own_global_pml) {
      if (i == 0) a.o0 = 0;
      if (i == nb - 1) a.o1 = n;
    }
    out[i] = a;
    int lo = i == 0 ? 0 : c[i], hi = i == nb - 1 ? n : c[i + 1];
    for (int g = lo; g < hi; ++g) near[g] = i;
  }
  return HD_OK;
}

constexpr int kMaxBoxWidth = 256;

}  // namespace hd

using namespace hd;

extern "C" {

const char *hd_last_error(void) { return g_err.c_str(); }

const char *hd_version(void) { return "hd 0.1 (sm_103a)"; }

int hd_setup_medium(hd_ctx **out, const hd_grid *grid, const hd_decomp *dec, const double *c_dev, int32_t precision,
                    void *stream) {
  if (!out) return invalid("hd_setup_medium: out is NULL");
  *out = nullptr;
  if (!grid || !dec || !c_dev) return invalid("hd_setup_medium: NULL argument");
  if (grid->nx < 1 || grid->ny < 1 || grid->npml < 0 || !(grid->h > 0) || !(grid->omega > 0) || grid->pml_power < 0 ||
      grid->pml_power > 8 || !std::isfinite(grid->sigma0_over_omega))
    return invalid("hd_setup_medium: bad grid");
  if (dec->nbx < 1 || dec->nby < 1 || dec->overlap < 0 || dec->nbx > grid->nx || dec->nby > grid->ny)
    return invalid("hd_setup_medium: bad decomposition");
  const int base_prec = precision & 0xff;
  if ((base_prec != HD_C128 && base_prec != HD_C64 && base_prec != HD_C64_H && base_prec != HD_C64_B) ||
      (precision & ~(0xff | HD_SYMMETRIC | HD_TCORE | HD_TF32X3 | HD_SMOOTH)))
    return invalid("hd_setup_medium: bad precision");
  if ((precision & HD_TF32X3) && !(precision & HD_TCORE))
    return invalid("hd_setup_medium: HD_TF32X3 is a variant of HD_TCORE");
  if ((precision & HD_TCORE) && (base_prec != HD_C64 || (precision & HD_SYMMETRIC)))
    return invalid("hd_setup_medium: HD_TCORE needs HD_C64 and excludes HD_SYMMETRIC");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  hd_ctx *c = new (std::nothrow) hd_ctx();
  if (!c) { set_error("hd_setup_medium: host allocation failed"); return HD_ERR_OOM; }
  c->nx_in = grid->nx; c->ny_in = grid->ny; c->npml = grid->npml;
  c->NX = grid->nx + 2 * grid->npml; c->NY = grid->ny + 2 * grid->npml;
  c->h = grid->h; c->omega = grid->omega; c->s0 = grid->sigma0_over_omega; c->power = grid->pml_power;
  c->prec = base_prec;
  c->sym = (precision & HD_SYMMETRIC) != 0;
  c->tc = (precision & HD_TCORE) != 0;
  c->tc3 = (precision & HD_TF32X3) != 0;
  c->smooth = (precision & HD_SMOOTH) != 0;
  c->stream = st;
  c->nbx = dec->nbx; c->nby = dec->nby; c->overlap = dec->overlap; c->own_global_pml = dec->own_global_pml ? 1 : 0;
  std::vector<int32_t> nearx, neary;
  int rc = axis_ranges(grid->nx, grid->npml, dec->nbx, dec->overlap, dec->cut_x, c->own_global_pml, c->axx, nearx, "x");
  if (!rc) rc = axis_ranges(grid->ny, grid->npml, dec->nby, dec->overlap, dec->cut_y, c->own_global_pml, c->axy, neary, "y");
  if (rc) { free_ctx(c); return rc; }
  c->nsub = c->nbx * c->nby;
  c->subs.resize(c->nsub);
  int64_t foff = 0, soff = 0, woff = 0;
  int32_t aoff = 0;
  c->max_m = 0; c->max_rows = 0;
  for (int iy = 0; iy < c->nby; ++iy)
    for (int ix = 0; ix < c->nbx; ++ix) {
      SubDev &s = c->subs[iy * c->nbx + ix];
      const AxisDev &ax = c->axx[ix], &ay = c->axy[iy];
      s.ex0 = ax.e0; s.ex = ax.e1 - ax.e0; s.ey0 = ay.e0; s.ey = ay.e1 - ay.e0;
      s.ox0 = ax.o0; s.ox1 = ax.o1; s.oy0 = ay.o0; s.oy1 = ay.o1;
      s.ix = ix; s.iy = iy;
      s.ldm = (s.ex + 3) & ~3;
      s.pad_ = 0;
      const int64_t mt = (s.ex + 15) / 16;
      const int64_t mp8 = (s.ex + 7) & ~7;
      s.foff = foff;
      foff += c->sym ? (int64_t)s.ey * (mt * (mt + 1) / 2) * 256
                     : (c->tc ? (c->tc3 ? 2 : 1) * (int64_t)s.ey * mp8 * mp8 : (int64_t)s.ey * s.ex * s.ldm);
      s.soff = soff; soff += (int64_t)s.ex * s.ey;
      s.woff = woff; woff += 2 * (int64_t)s.ex * s.ex;
      s.aoff = aoff; aoff += 2 * s.ex + 2 * s.ey + 2;
      c->max_m = std::max(c->max_m, s.ex);
      c->max_rows = std::max(c->max_rows, s.ey);
    }
  if (c->max_m > kMaxBoxWidth) {
    free_ctx(c);
    return invalid("hd_setup_medium: a box is wider than 256 cells (use more boxes along x)");
  }
  if (c->tc3 && c->max_m > kMaxBoxWidthX3) {
    free_ctx(c);
    return invalid("hd_setup_medium: HD_TF32X3 takes boxes up to 176 cells wide (use more boxes along x)");
  }
  c->factor_elems = foff; c->staging_elems = soff; c->work_elems = woff;
  const int64_t n = (int64_t)c->NX * c->NY;
#define ALLOC(p, bytes)                                                     \
  do {                                                                      \
    cudaError_t e_ = cudaMallocAsync((void **)&(p), (bytes), st);          \
    if (e_ != cudaSuccess) { free_ctx(c); return cuda_fail(e_, "cudaMallocAsync"); } \
  } while (0)
  ALLOC(c->d_k2, sizeof(double) * n);
  ALLOC(c->d_cc, sizeof(double) * n);
  ALLOC(c->d_gax_c, sizeof(double2) * c->NX);
  ALLOC(c->d_giax_f, sizeof(double2) * (c->NX + 1));
  ALLOC(c->d_gay_c, sizeof(double2) * c->NY);
  ALLOC(c->d_giay_f, sizeof(double2) * (c->NY + 1));
  ALLOC(c->d_lpool, sizeof(double2) * aoff);
  ALLOC(c->d_subs, sizeof(SubDev) * c->nsub);
  ALLOC(c->d_axx, sizeof(AxisDev) * c->nbx);
  ALLOC(c->d_axy, sizeof(AxisDev) * c->nby);
  ALLOC(c->d_nearx, sizeof(int32_t) * c->NX);
  ALLOC(c->d_neary, sizeof(int32_t) * c->NY);
  ALLOC(c->d_status, sizeof(int32_t));
  ALLOC(c->d_fflag, sizeof(int32_t) * c->nsub);
#undef ALLOC
  cudaError_t e;
#define CP(dst, src, bytes)                                                                        \
  do {                                                                                             \
    cudaError_t e_ = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, st);           \
    if (e_ != cudaSuccess) { free_ctx(c); return cuda_fail(e_, "cudaMemcpyAsync"); }               \
  } while (0)
  CP(c->d_subs, c->subs.data(), sizeof(SubDev) * c->nsub);
  CP(c->d_axx, c->axx.data(), sizeof(AxisDev) * c->nbx);
  CP(c->d_axy, c->axy.data(), sizeof(AxisDev) * c->nby);
  CP(c->d_nearx, nearx.data(), sizeof(int32_t) * c->NX);
  CP(c->d_neary, neary.data(), sizeof(int32_t) * c->NY);
#undef CP
  e = cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_fflag, 0, sizeof(int32_t) * c->nsub, st);
  if (e == cudaSuccess) e = launch_setup_tables(c, c_dev, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "hd_setup_medium"); }
  int32_t status = 0;
  e = cudaMemcpy(&status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "hd_setup_medium status"); }
  if (status) { free_ctx(c); set_error("hd_setup_medium: velocity must be finite and positive"); return HD_ERR_NUMERIC; }
  c->t_launch[T_OTHER] += 3;  // the three table kernels above
  lookup_tuning(c);   // a launch shape tuned earlier in this process for the same shape class
  *out = c;
  return HD_OK;
}

int hd_query_workspace(const hd_ctx *c, int32_t nrhs, int32_t restart, size_t *factor_bytes, size_t *krylov_bytes_out,
                       size_t *scratch_bytes) {
  if (nrhs < 1 || restart < 1 || restart > HD_MAX_RESTART)
    return invalid("hd_query_workspace: nrhs must be >= 1 and restart in 1 .. HD_MAX_RESTART");
  if (!c) return invalid("hd_query_workspace: NULL context");
  const size_t cs = compute_bytes(c->prec);
  if (factor_bytes) *factor_bytes = store_bytes(c->prec) * (size_t)c->factor_elems;
  if (scratch_bytes) *scratch_bytes = cs * (size_t)std::max(c->staging_elems * (int64_t)nrhs, c->work_elems);
  if (krylov_bytes_out) *krylov_bytes_out = krylov_bytes((int64_t)c->NX * c->NY, restart, nrhs);
  return HD_OK;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int hd_factor_subdomains(hd_ctx *c, void *factor, size_t factor_bytes, void *scratch, size_t scratch_bytes,
                         void *stream) {
  if (!c || !factor || !scratch) return invalid("hd_factor_subdomains: NULL argument");
  size_t fb, sb;
  hd_query_workspace(c, 1, 1, &fb, nullptr, &sb);
  if (factor_bytes < fb) { set_error("hd_factor_subdomains: factor workspace too small"); return HD_ERR_OOM; }
  if (scratch_bytes < sb) { set_error("hd_factor_subdomains: scratch workspace too small"); return HD_ERR_OOM; }
  if (!aligned16(factor) || !aligned16(scratch)) return invalid("hd_factor_subdomains: buffers must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = run_factor(c, factor, scratch, st);
  if (rc) return rc;
  c->factor = factor;
  c->factored = true;
  return HD_OK;
}

int hd_set_factor_path(hd_ctx *c, int32_t path, double pivot_ratio) {
  if (!c) return invalid("hd_set_factor_path: NULL context");
  if (path != HD_FACTOR_AUTO && path != HD_FACTOR_SIMT && path != HD_FACTOR_TCORE)
    return invalid("hd_set_factor_path: unknown path");
  if (!(pivot_ratio > 0) || !std::isfinite(pivot_ratio)) return invalid("hd_set_factor_path: pivot_ratio must be > 0");
  c->fpath = path;
  c->fpivot = pivot_ratio;
  return HD_OK;
}

int hd_factor_report(hd_ctx *c, int32_t *tcore_boxes, int32_t *pivoted_boxes, void *stream) {
  if (!c) return invalid("hd_factor_report: NULL context");
  if (c->last_fpath < 0) return invalid("hd_factor_report: no factorisation yet");
  int32_t tcb = 0, piv = c->nsub;
  if (c->last_fpath == HD_FACTOR_TCORE) {
    std::vector<int32_t> fl(c->nsub);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(fl.data(), c->d_fflag, sizeof(int32_t) * c->nsub, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "hd_factor_report");
    piv = 0;
    for (int32_t f : fl) piv += f != 0;
    tcb = c->nsub - piv;
  }
  if (tcore_boxes) *tcore_boxes = tcb;
  if (pivoted_boxes) *pivoted_boxes = piv;
  return HD_OK;
}

int hd_matvec(hd_ctx *c, const void *x, void *y, int32_t nrhs, void *stream) {
  if (!c || !x || !y || nrhs < 1) return invalid("hd_matvec: bad argument");
  if (!aligned16(x) || !aligned16(y)) return invalid("hd_matvec: vectors must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)c->NX * c->NY;
  tic(c, T_MATVEC, st);
  cudaError_t e = launch_matvec(c, reinterpret_cast<const double2 *>(x), n, reinterpret_cast<double2 *>(y), n, nrhs, st);
  toc(c, T_MATVEC, st, 1);
  if (e != cudaSuccess) return cuda_fail(e, "hd_matvec");
  return HD_OK;
}

int hd_rhs_from_source(hd_ctx *c, const void *f, void *b, int32_t nrhs, void *stream) {
  if (!c || !f || !b || nrhs < 1) return invalid("hd_rhs_from_source: bad argument");
  if (!aligned16(f) || !aligned16(b)) return invalid("hd_rhs_from_source: vectors must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)c->NX * c->NY;
  for (int r = 0; r < nrhs; ++r) {
    cudaError_t e = launch_rhs(c, reinterpret_cast<const double2 *>(f) + r * n, reinterpret_cast<double2 *>(b) + r * n, st);
    c->t_launch[T_OTHER] += 1;
    if (e != cudaSuccess) return cuda_fail(e, "hd_rhs_from_source");
  }
  return HD_OK;
}

int hd_apply_precond(hd_ctx *c, const void *r, void *z, int32_t nrhs, void *scratch, size_t scratch_bytes,
                     void *stream) {
  if (!c || !r || !z || !scratch || nrhs < 1) return invalid("hd_apply_precond: bad argument");
  if (!c->factored) return invalid("hd_apply_precond: call hd_factor_subdomains first");
  const size_t per = compute_bytes(c->prec) * (size_t)c->staging_elems;
  if (scratch_bytes < per) { set_error("hd_apply_precond: scratch workspace too small"); return HD_ERR_OOM; }
  if (!aligned16(r) || !aligned16(z) || !aligned16(scratch)) return invalid("hd_apply_precond: buffers must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)c->NX * c->NY;
  const int group = (int)std::min<size_t>((size_t)nrhs, scratch_bytes / per);   // right-hand sides per launch
  for (int k = 0; k < nrhs; k += group) {
    const int g = std::min(group, nrhs - k);
    int rc = run_apply(c, reinterpret_cast<const double2 *>(r) + k * n, n, reinterpret_cast<double2 *>(z) + k * n, n, g,
                       scratch, st);
    if (rc) return rc;
  }
  return HD_OK;
}

int hd_apply_ddm(hd_ctx *c, const void *f, void *u, int32_t nrhs, int32_t nsteps, void *work, size_t work_bytes,
                 void *scratch, size_t scratch_bytes, void *stream) {
  if (!c || !f || !u || !work || !scratch || nrhs < 1 || nsteps < 1) return invalid("hd_apply_ddm: bad argument");
  if (f == u) return invalid("hd_apply_ddm: u must not alias f");
  if (!c->factored) return invalid("hd_apply_ddm: call hd_factor_subdomains first");
  const int64_t n = (int64_t)c->NX * c->NY;
  if (work_bytes < 2 * sizeof(double2) * (size_t)n * nrhs) {
    set_error("hd_apply_ddm: work buffer too small (2 * nrhs * NX * NY * 16 bytes)");
    return HD_ERR_OOM;
  }
  if (scratch_bytes < compute_bytes(c->prec) * (size_t)c->staging_elems * nrhs) {
    set_error("hd_apply_ddm: scratch workspace too small for nrhs right-hand sides");
    return HD_ERR_OOM;
  }
  if (!aligned16(f) || !aligned16(u) || !aligned16(work) || !aligned16(scratch))
    return invalid("hd_apply_ddm: buffers must be 16-byte aligned");
  return run_apply_steps(c, reinterpret_cast<const double2 *>(f), n, reinterpret_cast<double2 *>(u), n, nrhs, nsteps,
                         reinterpret_cast<double2 *>(work), scratch, reinterpret_cast<cudaStream_t>(stream));
}

int hd_gmres_solve(hd_ctx *c, const void *b, void *x, int32_t nrhs, const hd_gmres_opts *o, void *kws, size_t kbytes,
                   void *scratch, size_t scratch_bytes, hd_gmres_stats *stats, void *stream) {
  if (!o) return invalid("hd_gmres_solve: bad argument");
  if (o->restart < 1 || o->restart > HD_MAX_RESTART || o->max_iters < 0 || !(o->rtol >= 0) ||
      (o->arnoldi != HD_ARNOLDI_FP64 && o->arnoldi != HD_ARNOLDI_DS) || (o->reorth != 0 && o->reorth != 1) ||
      o->precond_steps < 0 || o->precond_steps > 64)
    return invalid("hd_gmres_solve: bad options");
  if (!c || !b || !x || !kws || !scratch || !stats || nrhs < 1) return invalid("hd_gmres_solve: bad argument");
  if (!c->factored) return invalid("hd_gmres_solve: call hd_factor_subdomains first");
  size_t kb, sb;
  hd_query_workspace(c, nrhs, o->restart, nullptr, &kb, &sb);
  if (kbytes < kb) { set_error("hd_gmres_solve: krylov workspace too small for nrhs right-hand sides"); return HD_ERR_OOM; }
  if (scratch_bytes < sb) { set_error("hd_gmres_solve: scratch workspace too small for nrhs right-hand sides"); return HD_ERR_OOM; }
  if (!aligned16(b) || !aligned16(x) || !aligned16(kws) || !aligned16(scratch))
    return invalid("hd_gmres_solve: buffers must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::memset(stats, 0, sizeof(hd_gmres_stats) * nrhs);
  int rc = run_gmres_batch(c, reinterpret_cast<const double2 *>(b), reinterpret_cast<double2 *>(x), nrhs, o, kws,
                           scratch, stats, st);
  if (rc == HD_ERR_CUDA) return rc;
  int32_t status = 0;
  cudaError_t e = cudaMemcpyAsync(c->host_stat.data(), c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "hd_gmres_solve status");
  std::memcpy(&status, c->host_stat.data(), sizeof(int32_t));
  if (status & ST_TIMEOUT) { set_error("hd_gmres_solve: a bounded device wait gave up"); return HD_ERR_TIMEOUT; }
  if (status) { set_error("hd_gmres_solve: a zero pivot or non-finite value was flagged on the device"); return HD_ERR_NUMERIC; }
  if (rc == HD_ERR_NOT_CONVERGED) set_error("hd_gmres_solve: not converged within max_iters");
  if (rc == HD_ERR_NUMERIC) set_error("hd_gmres_solve: non-finite value in the Arnoldi process");
  return rc;
}

int hd_autotune(hd_ctx *c, const void *r, void *z, void *scratch, size_t scratch_bytes, int32_t *threads_out,
                int32_t *stages_out, float *ms_out, void *stream) {
  if (!c || !r || !z || !scratch) return invalid("hd_autotune: bad argument");
  if (!c->factored) return invalid("hd_autotune: call hd_factor_subdomains first");
  const size_t per = compute_bytes(c->prec) * (size_t)c->staging_elems;
  if (scratch_bytes < per) { set_error("hd_autotune: scratch workspace too small"); return HD_ERR_OOM; }
  int ct = 0, ns = 0;
  int rc = autotune_subst(c, reinterpret_cast<const double2 *>(r), reinterpret_cast<double2 *>(z), scratch,
                          reinterpret_cast<cudaStream_t>(stream), &ct, &ns, ms_out);
  if (threads_out) *threads_out = ct;
  if (stages_out) *stages_out = ns;
  return rc;
}

int hd_set_profiling(hd_ctx *c, int32_t on) {
  if (!c) return invalid("hd_set_profiling: NULL context");
  c->profiling = on != 0;
  return HD_OK;
}

int hd_get_timers(hd_ctx *c, double *ms, int64_t *launches, int32_t n, int32_t reset, void *stream) {
  if (!c) return invalid("hd_get_timers: NULL context");
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "hd_get_timers");
  collect_timers(c);
  for (int i = 0; i < n && i < T_NCLASS; ++i) {
    if (ms) ms[i] = c->t_ms[i];
    if (launches) launches[i] = c->t_launch[i];
  }
  if (reset)
    for (int i = 0; i < T_NCLASS; ++i) { c->t_ms[i] = 0; c->t_launch[i] = 0; }
  return HD_OK;
}

int hd_check_status(hd_ctx *c, int32_t clear, void *stream) {
  if (!c) return invalid("hd_check_status: NULL context");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(c->host_stat.data(), c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "hd_check_status");
  int32_t status;
  std::memcpy(&status, c->host_stat.data(), sizeof(int32_t));
  if (clear) {
    e = cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "hd_check_status clear");
  }
  if (status & ST_TIMEOUT) { set_error("device wait gave up"); return HD_ERR_TIMEOUT; }
  if (status) { set_error("zero pivot or non-finite value flagged on the device"); return HD_ERR_NUMERIC; }
  return HD_OK;
}

int hd_destroy(hd_ctx *c) {
  if (!c) return HD_OK;
  free_ctx(c);   // stream-ordered frees after the work queued on the set-up stream
  return HD_OK;
}

}  // extern "C"
