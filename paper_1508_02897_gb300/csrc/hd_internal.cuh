// Internal declarations shared by the translation units of libhd.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hd.h"

namespace hd {

// ---------------------------------------------------------------- complex helpers
template <typename R> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename R> using C = typename cplx<R>::type;

template <typename T> __host__ __device__ __forceinline__ T mk(decltype(T::x) re, decltype(T::x) im) {
  T z; z.x = re; z.y = im; return z;
}
// Products are written with explicit round-to-nearest intrinsics so the
// compiler cannot contract them differently in different instantiations:
// every kernel variant (for example one or several right-hand sides per CTA)
// then rounds identically and results are bitwise reproducible.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return mk<T>(add_rn(a.x, b.x), add_rn(a.y, b.y)); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return mk<T>(add_rn(a.x, -b.x), add_rn(a.y, -b.y)); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return mk<T>(fma_rn(a.x, b.x, -mul_rn(a.y, b.y)), fma_rn(a.x, b.y, mul_rn(a.y, b.x)));
}
// acc + a*b
template <typename T> __device__ __forceinline__ T cfma(T a, T b, T acc) {
  acc.x = fma_rn(a.x, b.x, acc.x); acc.x = fma_rn(-a.y, b.y, acc.x);
  acc.y = fma_rn(a.x, b.y, acc.y); acc.y = fma_rn(a.y, b.x, acc.y);
  return acc;
}
// acc - a*b
template <typename T> __device__ __forceinline__ T cfms(T a, T b, T acc) {
  acc.x = fma_rn(-a.x, b.x, acc.x); acc.x = fma_rn(a.y, b.y, acc.x);
  acc.y = fma_rn(-a.x, b.y, acc.y); acc.y = fma_rn(-a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a)*b
template <typename T> __device__ __forceinline__ T cfma_conj(T a, T b, T acc) {
  acc.x = fma_rn(a.x, b.x, acc.x); acc.x = fma_rn(a.y, b.y, acc.x);
  acc.y = fma_rn(a.x, b.y, acc.y); acc.y = fma_rn(-a.y, b.x, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ T cinv(T a) {
  auto d = fma_rn(a.x, a.x, mul_rn(a.y, a.y));
  return mk<T>(a.x / d, -a.y / d);
}
// Scale of the first Gram-Schmidt pass's output in the double-single mode: 1 / ||w|| from
// the pass's self dot product ||w||^2 (1 when that is zero or not finite).  The stored
// vector then has the norm ||w - V h|| / ||w|| <= 1 whatever the norms of earlier ones, so
// lazily normalised magnitudes cannot compound over a restart cycle.
__host__ __device__ __forceinline__ double lazy_gamma(double w2) {
  return (w2 > 0.0 && w2 < 1.0e300) ? 1.0 / sqrt(w2) : 1.0;
}
// FP64 <-> float-pair conversions without conversion instructions, which on this GPU
// issue at the FP64 pipe's rate (1/64 of FP32).  ds_split(x) = (h, l): h is x truncated
// to 24 significant bits (its bits moved into float fields), l = x - h rounded to float.
// The 29 bits below h are turned into floats by the exponent trick: a float with
// exponent field E and mantissa field q is 2^(E-127) + q 2^(E-150), so subtracting
// 2^(E-127) leaves q 2^(E-150) exactly; the top 23 and the low 6 of the 29 bits each
// take one such subtraction and one rounded FP32 add joins them (|x - h - l| <= 2^-47
// |x|).  Valid for FP64 exponents 949..1150 (|x| in [2^-74, 2^128)), where every
// intermediate float is normal; zero and FP64 subnormals give (0, 0), everything else
// (tiny, huge, inf, NaN) takes the conversion instructions.
__device__ __forceinline__ float2 ds_split(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const unsigned int e = (hi >> 20) & 0x7FFu;
  if (e - 949u > 1150u - 949u) {
    if (e == 0u) return make_float2(0.f, 0.f);
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
  }
  const unsigned int sg = hi & 0x80000000u;
  const unsigned int eh = (e - 896u) << 23;                                  // float exponent field of h
  const float h = __uint_as_float(sg | eh | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu));
  const unsigned int e1 = sg | (eh - (23u << 23)), e0 = sg | (eh - (29u << 23));
  const float l1 = __fsub_rn(__uint_as_float(e1 | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(e1));
  const float l0 = __fsub_rn(__uint_as_float(e0 | (lo & 63u)), __uint_as_float(e0));
  return make_float2(h, __fadd_rn(l1, l0));
}
// float -> FP64 by moving the fields (exact); zero gives 0, subnormals, inf and NaN convert.
__device__ __forceinline__ double ds_f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e - 1u > 253u) return (u << 1) == 0u ? 0.0 : (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
}
// h + l in FP64: one FP64 add.
__device__ __forceinline__ double ds_to_d(float h, float l) { return ds_f2d(h) + ds_f2d(l); }
// (sh, sl) += (ah + al)(bh + bl), error-free hi product, FP32 cross terms.
__device__ __forceinline__ void ds_mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
  float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  float t = __fadd_rn(sh, p);
  float z = __fsub_rn(t, sh);
  float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ void ds_renorm(float &sh, float &sl) {
  float t = __fadd_rn(sh, sl);
  sl = __fsub_rn(sl, __fsub_rn(t, sh));
  sh = t;
}

__device__ __forceinline__ void ds_add(float &sh, float &sl, float bh, float bl) {
  float t = __fadd_rn(sh, bh);
  float z = __fsub_rn(t, sh);
  float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(bh, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, bl));
  ds_renorm(sh, sl);
}
__host__ __device__ __forceinline__ float2 to_c(double2 z, float2) { return make_float2((float)z.x, (float)z.y); }
__host__ __device__ __forceinline__ double2 to_c(double2 z, double2) { return z; }
__host__ __device__ __forceinline__ double2 to_d(float2 z) { return make_double2(z.x, z.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 z) { return z; }

// Stored factor entries: the compute type itself, or complex FP16 / BF16 for FP32 math.
template <typename S, typename T> __device__ __forceinline__ S store_c(T v) { return v; }
template <> __device__ __forceinline__ __half2 store_c<__half2, float2>(float2 v) { return __float22half2_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat162 store_c<__nv_bfloat162, float2>(float2 v) {
  return __float22bfloat162_rn(v);
}
template <typename T, typename S> __device__ __forceinline__ T load_c(S v) { return v; }
template <> __device__ __forceinline__ float2 load_c<float2, __half2>(__half2 v) { return __half22float2(v); }
template <> __device__ __forceinline__ float2 load_c<float2, __nv_bfloat162>(__nv_bfloat162 v) {
  return __bfloat1622float2(v);
}

// Bytes of one stored factor entry and of one compute (staging / working) entry.
inline size_t store_bytes(int prec) { return prec == HD_C128 ? 16 : (prec == HD_C64 ? 8 : 4); }
inline size_t compute_bytes(int prec) { return prec == HD_C128 ? 16 : 8; }

// Entries of D_j (tridiagonal) and the coupling L_j of grid row j, Eq. (pml)
// discretised with the box's own PML tables.
template <typename T, typename R>
__device__ __forceinline__ T d_entry(int r, int c, int j, const double2 *a1c, const double2 *ia1f, const double2 *a2c,
                                     const double2 *ia2f, const double *k2row, double h2) {
  const double2 a2 = a2c[j];
  if (r == c) {
    const double2 a1 = a1c[r];
    const double2 cw = cmul(a2, ia1f[r]), ce = cmul(a2, ia1f[r + 1]);
    const double2 cs = cmul(a1, ia2f[j]), cn = cmul(a1, ia2f[j + 1]);
    const double2 j12 = cmul(a1, a2);
    const double hk = mul_rn(h2, k2row[r]);
    return mk<T>((R)(-(cw.x + ce.x + cs.x + cn.x) + hk * j12.x), (R)(-(cw.y + ce.y + cs.y + cn.y) + hk * j12.y));
  }
  if (r == c + 1) {
    const double2 cw = cmul(a2, ia1f[r]);      // row r couples to column r-1 (west)
    return mk<T>((R)cw.x, (R)cw.y);
  }
  if (r + 1 == c) {
    const double2 ce = cmul(a2, ia1f[r + 1]);  // row r couples to column r+1 (east)
    return mk<T>((R)ce.x, (R)ce.y);
  }
  return mk<T>(0, 0);
}

// d_entry restricted to its tridiagonal band (zero elsewhere without touching the tables)
template <typename T, typename R>
__device__ __forceinline__ T d_band(int r, int c, int j, const double2 *a1c, const double2 *ia1f, const double2 *a2c,
                                    const double2 *ia2f, const double *k2row, double h2) {
  return (r - c <= 1 && c - r <= 1) ? d_entry<T, R>(r, c, j, a1c, ia1f, a2c, ia2f, k2row, h2) : mk<T>(0, 0);
}

// Storage layouts of the S_j^{-1}: full column-major blocks, upper 16 x 16 tiles,
// or TF32 real/imaginary planes in the tensor-core operand layout (HD_TCORE).
// LAY_TC3: the same layout with four planes per chunk (real hi, imaginary hi, real lo,
// imaginary lo), hi = TF32 rounding and lo = TF32 rounding of the remainder (HD_TF32X3).
enum { LAY_FULL = 0, LAY_SYM = 1, LAY_TC = 2, LAY_TC3 = 3 };

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------- tables
// One overlapping box Omega_ij (global cell indices) and its owned box.
struct SubDev {
  int32_t ex0, ey0, ex, ey;      // extent origin and size
  int32_t ox0, ox1, oy0, oy1;    // owned box [ox0, ox1) x [oy0, oy1)
  int64_t foff;                  // offset of the factors (complex entries)
  int64_t soff;                  // offset of the staging vector (complex entries)
  int64_t woff;                  // offset of the factorisation working matrix (complex entries)
  int32_t aoff;                  // offset into the local PML table pool
  int32_t ix, iy;
  int32_t ldm;                   // leading dimension of a stored S_j^{-1} (m rounded up to a multiple of 4)
  int32_t pad_;
};

// One axis of the decomposition: per box column (or row) its extent and owned range.
struct AxisDev {
  int32_t e0, e1, o0, o1;
};

// A captured Arnoldi step (CUDA graph) and the kernels it holds per timer class.
struct GraphKey {
  const void *kws, *scratch, *factor;
  int B, R, mode, j, ct, ns;   // mode: bit 0 double-single Arnoldi, bit 1 selective reorthogonalisation,
                               // bits 2..: preconditioner steps
  bool operator<(const GraphKey &o) const {
    return std::tie(kws, scratch, factor, B, R, mode, j, ct, ns) <
           std::tie(o.kws, o.scratch, o.factor, o.B, o.R, o.mode, o.j, o.ct, o.ns);
  }
};

enum TimerClass { T_FACTOR = 0, T_SUBST = 1, T_GATHER = 2, T_MATVEC = 3, T_ARNOLDI = 4, T_OTHER = 5, T_NCLASS = 6 };

// Bits of the device status word.
enum StatusBits { ST_ZERO_PIVOT = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t kernels[T_NCLASS] = {0};
};

}  // namespace hd

struct hd_ctx {
  // grid
  int nx_in, ny_in, npml, NX, NY;
  double h, omega, s0;
  int power;
  int prec;
  bool sym = false;   // S_j^{-1} stored as upper 16 x 16 tiles (HD_SYMMETRIC)
  bool tc = false;    // S_j^{-1} stored in the tensor-core operand layout (HD_TCORE)
  bool tc3 = false;   // ... as TF32 hi/lo pairs, FP32-grade products (HD_TF32X3)
  bool smooth = false;   // local solutions weighted by the smoothing function beta (HD_SMOOTH)
  // decomposition
  int nbx, nby, overlap, own_global_pml;
  int nsub;
  std::vector<hd::SubDev> subs;
  std::vector<hd::AxisDev> axx, axy;
  int max_m, max_rows;
  int64_t factor_elems, staging_elems, work_elems;
  // device tables (owned)
  double *d_k2 = nullptr;
  double *d_cc = nullptr;   // h^2 k^2 - 4: the centre coefficient of A outside the PML
  double2 *d_gax_c = nullptr, *d_giax_f = nullptr, *d_gay_c = nullptr, *d_giay_f = nullptr;
  double2 *d_lpool = nullptr;   // per-box PML tables: a1c[ex], ia1f[ex+1], a2c[ey], ia2f[ey+1]
  hd::SubDev *d_subs = nullptr;
  hd::AxisDev *d_axx = nullptr, *d_axy = nullptr;
  int32_t *d_nearx = nullptr, *d_neary = nullptr;  // per global index: box column/row nearest
  int32_t *d_status = nullptr;                    // device status word
  int32_t *d_fflag = nullptr;                     // per box: 1 if the tensor-core factorisation marked it
  int fpath = 0;                                  // hd_factor_path of hd_set_factor_path
  double fpivot = 0.5;                            // pivot ratio of the tensor-core factorisation's check
  int last_fpath = -1;                            // kernel of the last factorisation (1 SIMT, 2 tensor cores)
  cudaStream_t stream = nullptr;                  // set-up stream: the context's tables are freed on it
  std::vector<double> host_stat = std::vector<double>(8);   // host mirror of small device results
  std::vector<unsigned char> host_buf;            // per-solve host mirror (grows on demand)
  // factor binding
  void *factor = nullptr;
  bool factored = false;
  // substitution launch shape chosen by hd_autotune (0: built-in heuristic)
  int tune_ct = 0, tune_ns = 0;
  // captured Arnoldi steps (hd_gmres_opts.graphs), run on the context's own stream
  std::map<hd::GraphKey, hd::GraphEntry> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gevent = nullptr;
  // profiling
  bool profiling = false;
  double t_ms[hd::T_NCLASS] = {0};
  int64_t t_launch[hd::T_NCLASS] = {0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  size_t ev_next = 0;
};

namespace hd {
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
#define HD_CUDA(call)                                         \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::hd::cuda_fail(e_, #call); \
  } while (0)

// Dynamic shared memory: a kernel's limit is raised to the most the device allows it
// (the opt-in maximum less its static shared memory), the same value on every call.
// Server slots launch one kernel with different sizes from several host threads at once;
// a limit set to each launch's own size would race (one thread lowering it between
// another's set and launch).  Sizes above the device's maximum give cudaErrorInvalidValue.
cudaError_t allow_smem_ptr(const void *kernel, size_t bytes);
template <typename K> cudaError_t allow_smem(K *kernel, size_t bytes) {
  return allow_smem_ptr(reinterpret_cast<const void *>(kernel), bytes);
}

// profiling brackets around a launch on `st`
void tic(hd_ctx *ctx, int cls, cudaStream_t st);
void toc(hd_ctx *ctx, int cls, cudaStream_t st, int nkernels);
int collect_timers(hd_ctx *ctx);

// kernels launchers (return cudaError_t of the launch)
cudaError_t launch_setup_tables(hd_ctx *ctx, const double *c_dev, cudaStream_t st);
cudaError_t launch_matvec(hd_ctx *ctx, const double2 *x, int64_t xs, double2 *y, int64_t ys, int nrhs,
                          cudaStream_t st);
cudaError_t launch_residual(hd_ctx *ctx, const double2 *b, const double2 *x, double2 *r, int nrhs, cudaStream_t st);
cudaError_t launch_rhs(hd_ctx *ctx, const double2 *f, double2 *b, cudaStream_t st);
int run_factor(hd_ctx *ctx, void *factor, void *work, cudaStream_t st);
// z = M r for nrhs vectors (r and z strided by rs and zs complex entries); the
// staging buffer holds nrhs per-RHS staging vectors of staging_elems entries.
int run_apply(hd_ctx *ctx, const double2 *r, int64_t rs, double2 *z, int64_t zs, int nrhs, void *staging,
              cudaStream_t st);
// z = sum over nsteps of the multi-step DDM (residual correction around run_apply);
// work holds 2 * nrhs vectors of NX*NY (residual, correction).
int run_apply_steps(hd_ctx *ctx, const double2 *r, int64_t rs, double2 *z, int64_t zs, int nrhs, int nsteps,
                    double2 *work, void *staging, cudaStream_t st);
// r = b - A x with strided vectors (nrhs on grid.z)
cudaError_t launch_residual_strided(hd_ctx *ctx, const double2 *b, int64_t bs, const double2 *x, int64_t xs,
                                    double2 *r, int64_t rs, int nrhs, cudaStream_t st);
// Restrict + forward/back substitution on the tensor cores (HD_TCORE storage), staging out.
cudaError_t launch_subst_tc(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vec_stride, void *staging,
                            int64_t stg_stride, cudaStream_t st);
// The FP32-grade tensor-core substitution (hd_subst_x3.cu, storage HD_TCORE | HD_TF32X3).
constexpr int kMaxBoxWidthX3 = 176;
cudaError_t launch_subst_x3(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vec_stride, void *staging,
                            int64_t stg_stride, cudaStream_t st);
size_t krylov_bytes(int64_t n, int restart, int nrhs);
bool lookup_tuning(hd_ctx *ctx);
int autotune_subst(hd_ctx *ctx, const double2 *r, double2 *z, void *staging, cudaStream_t st, int *ct_out,
                   int *ns_out, float *ms_out);
int run_gmres_batch(hd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const hd_gmres_opts *o, void *kws,
                    void *scratch, hd_gmres_stats *stats, cudaStream_t st);
// Streaming double-single Gram-Schmidt passes (hd_gs.cu).  gs_items(n): work items (and
// partial sums) per right-hand side; the dots take at most kGsDotsMax basis vectors.
constexpr int kGsDotsMax = 12;
int gs_items(int64_t n);
cudaError_t launch_gs_dots(const float4 *V, int64_t ldv, int64_t ldvr, int nk0, const double2 *w, int64_t ldw,
                           int64_t n, int B, double2 *partial, int64_t ldp, const int *skip, const int *live, int self,
                           int32_t *status, cudaStream_t st);
cudaError_t launch_gs_update(const float4 *V, int64_t ldv, int64_t ldvr, int nk, const double2 *coef, int ldc,
                             const double *sc, const double2 *base, double2 *y, int64_t ldy, float4 *vout, int64_t n,
                             int B, double2 *normpart, int64_t ldp, const int *skip, const int *live, int scale,
                             int32_t *status, cudaStream_t st);
size_t factor_smem_bytes(int prec, int max_m);
// Block flexible GMRES (hd_block.cu)
size_t block_krylov_bytes(int64_t n, int restart, int p);
int run_block_gmres(hd_ctx *ctx, const double2 *b, double2 *x, int p, const hd_gmres_opts *o, void *kws,
                    void *scratch, hd_gmres_stats *stats, cudaStream_t st);
// Tensor-core factorisation (hd_factor_tc.cu): complex FP32 arithmetic, boxes up to 192 wide.
bool factor_tc_supported(const hd_ctx *ctx);
cudaError_t launch_factor_tc(hd_ctx *ctx, void *factor, cudaStream_t st);
size_t factor_tc_smem_bytes();
}  // namespace hd
