// Preconditioner application that allocates nothing: the staging vectors of
// the local substitutions live in a fixed device array of this file.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "hd_internal.cuh"

// ---------------------------------------------------------------------------
// Preconditioner application without any allocation.
//
// Some callers cannot call cudaMalloc when they apply the preconditioner:
// plug-ins whose host application owns the device heap through its own pool,
// latency-bound loops where an allocation could synchronise the device, and
// long-running services that must keep a fixed device footprint after
// start-up.  For them the staging vectors live in one fixed device array
// inside this library.  In host code the array's name is only a host-side
// stand-in, so its device address is looked up (cudaGetSymbolAddress, with the
// device current) the first time a call runs in a given CUDA context, and
// passed to the kernels.  The lookup is remembered per context (device and
// driver context handle), so a device reset or a caller-made context gets a
// fresh lookup instead of a stale address.  Every GPU that loads the library
// holds the array until the process exits.
namespace hd {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
// remembered lookups: (device, context handle) -> address
struct StaticEntry {
  int dev;
  void *ctx;
  void *ptr;
};
static std::vector<StaticEntry> g_static_cache;

// The current driver context handle, through the runtime's driver entry point (the
// library links the CUDA runtime only); nullptr if it cannot be had.
static void *current_context() {
  typedef int (*GetCurrentFn)(void **);
  static GetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCurrentFn>(f);
  }
  void *ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

static int static_scratch_ptr(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_static_mu);
  void *ctx = current_context();
  if (ctx)
    for (const StaticEntry &se : g_static_cache)
      if (se.dev == dev && se.ctx == ctx) {
        *out = se.ptr;
        return HD_OK;
      }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
  if (ctx) g_static_cache.push_back({dev, ctx, p});   // without a handle: look up on every call
  *out = p;
  return HD_OK;
}

}  // namespace hd

extern "C" int hd_apply_precond_noalloc(hd_ctx *c, const void *r, void *z, int32_t nrhs, void *stream) {
  using namespace hd;
  if (!c || !r || !z || nrhs < 1) { set_error("hd_apply_precond_noalloc: bad argument"); return HD_ERR_INVALID; }
  if ((reinterpret_cast<uintptr_t>(r) & 15) || (reinterpret_cast<uintptr_t>(z) & 15)) {
    set_error("hd_apply_precond_noalloc: vectors must be 16-byte aligned");
    return HD_ERR_INVALID;
  }
  const size_t cs = compute_bytes(c->prec);
  const size_t need = cs * (size_t)c->staging_elems;   // one right-hand side
  if (need > kStaticScratchBytes) {
    set_error("hd_apply_precond_noalloc: the staging vectors need " + std::to_string(need) +
              " bytes, more than the library's fixed 64 MiB array; use hd_apply_precond with a caller workspace");
    return HD_ERR_OOM;
  }
  if (!c->factored) { set_error("hd_apply_precond_noalloc: call hd_factor_subdomains first"); return HD_ERR_INVALID; }
  void *scratch = nullptr;
  int rc = static_scratch_ptr(&scratch);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)c->NX * c->NY;
  const int group = (int)std::min<size_t>((size_t)nrhs, kStaticScratchBytes / need);
  for (int k = 0; k < nrhs; k += group) {
    const int g = std::min(group, nrhs - k);
    rc = run_apply(c, reinterpret_cast<const double2 *>(r) + k * n, n, reinterpret_cast<double2 *>(z) + k * n, n, g,
                   scratch, st);
    if (rc) return rc;
  }
  return HD_OK;
}

