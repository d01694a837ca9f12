// Preconditioner application that allocates nothing: the staging vectors of
// the local substitutions live in a fixed device array of this file.
#include <algorithm>
#include <mutex>
#include <string>

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
// stand-in, so its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current, on the first call made on
// that device) and passed to the kernels.  Every GPU that loads the library
// holds the array until the process exits.
namespace hd {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[64] = {nullptr};

static int static_scratch_ptr(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) { set_error("device index out of range"); return HD_ERR_INVALID; }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
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

