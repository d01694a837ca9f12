// Throughput probes used as roofline denominators: FP64 and FP32 FMA rates
// (eight independent chains per thread) and a device-to-device copy.
#include "hd_internal.cuh"

namespace hd {

template <typename T>
__global__ void k_probe_fma(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

__global__ void k_probe_copy(const float4 *__restrict__ a, float4 *__restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

}  // namespace hd

extern "C" int hd_probe_peaks(void *buf_dev, size_t buf_bytes, double *fp64_tflops, double *fp32_tflops,
                              double *copy_gbs, void *stream) {
  using namespace hd;
  if (!buf_dev || buf_bytes < ((size_t)64 << 20)) { set_error("hd_probe_peaks: need a buffer of at least 64 MiB"); return HD_ERR_INVALID; }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  auto timed = [&](auto launch) {
    launch();  // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms;
  };
  const int it64 = 2048, it32 = 32768;
  double t = timed([&] { k_probe_fma<double><<<blocks, threads, 0, st>>>((double *)buf_dev, it64, 0.999, 0.001); });
  if (fp64_tflops) *fp64_tflops = 2.0 * 32 * it64 * (double)blocks * threads / (t * 1e-3) / 1e12;
  t = timed([&] { k_probe_fma<float><<<blocks, threads, 0, st>>>((float *)buf_dev, it32, 0.999f, 0.001f); });
  if (fp32_tflops) *fp32_tflops = 2.0 * 32 * it32 * (double)blocks * threads / (t * 1e-3) / 1e12;
  const size_t half = (buf_bytes / 2) & ~(size_t)15, n = half / 16;
  t = timed([&] {
    k_probe_copy<<<sms * 16, 512, 0, st>>>((const float4 *)buf_dev, (float4 *)((char *)buf_dev + half), n);
  });
  if (copy_gbs) *copy_gbs = 2.0 * half / (t * 1e-3) / 1e9;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hd_probe_peaks");
  return HD_OK;
}
