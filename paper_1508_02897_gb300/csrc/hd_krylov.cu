// Outer Krylov loop (Sec. 3: restarted GMRES to a relative tolerance), FP64.
//
// Right-preconditioned flexible GMRES: Z_j = M v_j is stored so that
// x = x0 + Z y holds for the preconditioner as applied.  Arnoldi uses
// classical Gram-Schmidt applied twice (CGS2), in FP64 or in double-single
// arithmetic (HD_ARNOLDI_DS, below):
//     h = V^H w, w -= V h, h' = V^H w, w -= V h', h += h', v_{j+1} = w/||w||,
// then complex Givens rotations with real cosine update the least-squares
// right-hand side g, and the cycle stops once |g_{j+1}| <= rtol ||b||.  The
// FP64 true residual b - A x decides convergence at the end of each cycle.
//
// Kernels: k_dots (block partial sums of V^H w, w held in registers), k_reduce
// (fixed-order sum of the partials: deterministic), k_update (w = base + sgn V c,
// optionally with block partials of ||w||^2), and single-thread kernels for the
// O(restart) Hessenberg/Givens/triangular work.  The host reads 32 bytes per
// Arnoldi step to decide whether to stop.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "hd_internal.cuh"

namespace hd {

constexpr int DT = 256;           // threads per block of the vector kernels
constexpr int DE = 8;             // elements per thread
constexpr int DCHUNK = DT * DE;   // elements per block

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// partial[k*G + blk] = sum over the block's chunk of conj(V[k][i]) w[i], k < nk.
__global__ void __launch_bounds__(DT) k_dots(const double2 *__restrict__ V, int64_t ldv, int nk,
                                             const double2 *__restrict__ w, int64_t n,
                                             double2 *__restrict__ partial, int G) {
  extern __shared__ double2 red[];  // [DT/32][nk]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * DCHUNK + tid;
  double2 wv[DE];
#pragma unroll
  for (int e = 0; e < DE; ++e) {
    int64_t i = base + (int64_t)DT * e;
    wv[e] = i < n ? w[i] : make_double2(0.0, 0.0);
  }
  for (int k = 0; k < nk; ++k) {
    const double2 *vk = V + (int64_t)k * ldv;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < DE; ++e) {
      int64_t i = base + (int64_t)DT * e;
      if (i < n) acc = cfma_conj(vk[i], wv[e], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp * nk + k] = acc;
  }
  __syncthreads();
  for (int k = tid; k < nk; k += DT) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < DT / 32; ++q) s = cadd(s, red[q * nk + k]);
    partial[(int64_t)k * G + blockIdx.x] = s;
  }
}

// out[k] = sum_b partial[k*G + b] in a fixed order.
__global__ void __launch_bounds__(256) k_reduce(const double2 *__restrict__ partial, int G, double2 *__restrict__ out) {
  __shared__ double2 sm[256];
  const int k = blockIdx.x, tid = threadIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = tid; b < G; b += 256) acc = cadd(acc, partial[(int64_t)k * G + b]);
  sm[tid] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) sm[tid] = cadd(sm[tid], sm[tid + s]);
    __syncthreads();
  }
  if (tid == 0) out[k] = sm[0];
}

// y = base + sgn * sum_k V[k] coef[k]; optionally normpart[blk] = block sum of |y|^2.
template <bool NORM>
__global__ void __launch_bounds__(DT) k_update(const double2 *__restrict__ V, int64_t ldv, int nk,
                                               const double2 *__restrict__ coef, double sgn, const double2 *base,
                                               double2 *y, int64_t n, double2 *__restrict__ normpart) {
  extern __shared__ double2 cs[];  // [nk]
  __shared__ double nsm[DT / 32];
  const int tid = threadIdx.x;
  for (int k = tid; k < nk; k += DT) cs[k] = coef[k];
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * DCHUNK + tid;
  double2 acc[DE];
#pragma unroll
  for (int e = 0; e < DE; ++e) acc[e] = make_double2(0.0, 0.0);
  for (int k = 0; k < nk; ++k) {
    const double2 *vk = V + (int64_t)k * ldv;
    const double2 ck = cs[k];
#pragma unroll
    for (int e = 0; e < DE; ++e) {
      int64_t i = b0 + (int64_t)DT * e;
      if (i < n) acc[e] = cfma(vk[i], ck, acc[e]);
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int e = 0; e < DE; ++e) {
    int64_t i = b0 + (int64_t)DT * e;
    if (i < n) {
      double2 bv = base ? base[i] : make_double2(0.0, 0.0);
      double2 o = make_double2(bv.x + sgn * acc[e].x, bv.y + sgn * acc[e].y);
      y[i] = o;
      if (NORM) nrm += o.x * o.x + o.y * o.y;
    }
  }
  if (NORM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) nsm[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int q = 0; q < DT / 32; ++q) s += nsm[q];
      normpart[blockIdx.x] = make_double2(s, 0.0);
    }
  }
}

// v = w * (1/scale) with scale = sqrt(red->x) (a squared norm) or the host value.
__global__ void __launch_bounds__(256) k_scale(const double2 *__restrict__ w, const double2 *__restrict__ red,
                                               double host_scale, double2 *__restrict__ v, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = red ? sqrt(red->x) : host_scale;
  double inv = s > 0.0 ? 1.0 / s : 0.0;
  double2 a = w[i];
  v[i] = make_double2(a.x * inv, a.y * inv);
}

// ---------------------------------------------------------------- double-single Arnoldi
// GB300 runs FP64 at 1/61 of its FP32 rate, which makes an FP64 Gram-Schmidt
// ALU-bound.  In this mode the basis V is stored as pairs of floats (hi, lo)
// with hi + lo equal to the FP64 value to about 2^-48, and the dot products
// and updates use double-single arithmetic (Dekker/Knuth error-free products
// and sums on the FP32 pipes).  The FP64 copy of the newest basis vector feeds
// the preconditioner; the residuals, norms, Hessenberg and Givens work stay FP64.
constexpr int DFC = 4096;  // elements of w staged per block in k_dots_df

__device__ __forceinline__ float2 split_d(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

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

// partial[k*G + blk] = sum over the block's DFC elements of conj(V[k][i]) w[i].
__global__ void __launch_bounds__(256) k_dots_df(const float4 *__restrict__ V, int64_t ldv, int nk,
                                                 const double2 *__restrict__ w, int64_t n,
                                                 double2 *__restrict__ partial, int G) {
  extern __shared__ float4 wsm[];  // [DFC]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * DFC;
  const int cnt = (int)min((int64_t)DFC, n - base);
  for (int i = tid; i < DFC; i += 256) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < cnt) {
      double2 x = w[base + i];
      float2 r = split_d(x.x), m = split_d(x.y);
      v = make_float4(r.x, r.y, m.x, m.y);
    }
    wsm[i] = v;
  }
  __syncthreads();
  for (int k = warp; k < nk; k += 8) {
    const float4 *vk = V + (int64_t)k * ldv + base;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int i0 = 0; i0 < cnt; i0 += 256) {
      float4 vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        int i = i0 + u * 32 + lane;
        vv[u] = i < cnt ? vk[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 a = vv[u], b = wsm[i0 + u * 32 + lane];
        ds_mac(rh, rl, a.x, a.y, b.x, b.y);     // re += ar br
        ds_mac(rh, rl, a.z, a.w, b.z, b.w);     // re += ai bi
        ds_mac(ih, il, a.x, a.y, b.z, b.w);     // im += ar bi
        ds_mac(ih, il, -a.z, -a.w, b.x, b.y);   // im -= ai br
      }
      ds_renorm(rh, rl);
      ds_renorm(ih, il);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
      float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
      ds_add(rh, rl, a, b);
      ds_add(ih, il, c, d);
    }
    if (lane == 0) partial[(int64_t)k * G + blockIdx.x] = make_double2((double)rh + (double)rl, (double)ih + (double)il);
  }
}

// y = base - sum_k V[k] coef[k] (double-single accumulation, FP64 result);
// optionally normpart[blk] = block sum of |y|^2.
template <bool NORM>
__global__ void __launch_bounds__(DT) k_update_df(const float4 *__restrict__ V, int64_t ldv, int nk,
                                                  const double2 *__restrict__ coef, const double2 *base, double2 *y,
                                                  int64_t n, double2 *__restrict__ normpart) {
  extern __shared__ float4 csm[];  // [nk]
  __shared__ double nsm[DT / 32];
  const int tid = threadIdx.x;
  for (int k = tid; k < nk; k += DT) {
    double2 c = coef[k];
    float2 r = split_d(c.x), m = split_d(c.y);
    csm[k] = make_float4(r.x, r.y, m.x, m.y);
  }
  __syncthreads();
  constexpr int E = 4;
  const int64_t b0 = (int64_t)blockIdx.x * DCHUNK + tid;
  double nrm = 0.0;
#pragma unroll 1
  for (int half = 0; half < DE / E; ++half) {
    float rh[E], rl[E], ih[E], il[E];
#pragma unroll
    for (int e = 0; e < E; ++e) { rh[e] = rl[e] = ih[e] = il[e] = 0.f; }
    for (int k = 0; k < nk; ++k) {
      const float4 c = csm[k];
      const float4 *vk = V + (int64_t)k * ldv;
      float4 a[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        int64_t i = b0 + (int64_t)DT * (half * E + e);
        a[e] = i < n ? vk[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        ds_mac(rh[e], rl[e], a[e].x, a[e].y, c.x, c.y);      // re += ar cr
        ds_mac(rh[e], rl[e], -a[e].z, -a[e].w, c.z, c.w);    // re -= ai ci
        ds_mac(ih[e], il[e], a[e].x, a[e].y, c.z, c.w);      // im += ar ci
        ds_mac(ih[e], il[e], a[e].z, a[e].w, c.x, c.y);      // im += ai cr
      }
      if ((k & 7) == 7) {
#pragma unroll
        for (int e = 0; e < E; ++e) { ds_renorm(rh[e], rl[e]); ds_renorm(ih[e], il[e]); }
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      int64_t i = b0 + (int64_t)DT * (half * E + e);
      if (i < n) {
        double2 bv = base[i];
        double2 o = make_double2(bv.x - ((double)rh[e] + (double)rl[e]), bv.y - ((double)ih[e] + (double)il[e]));
        y[i] = o;
        if (NORM) nrm += o.x * o.x + o.y * o.y;
      }
    }
  }
  if (NORM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) nsm[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int q = 0; q < DT / 32; ++q) s += nsm[q];
      normpart[blockIdx.x] = make_double2(s, 0.0);
    }
  }
}

// v = w / scale written twice: split into V (double-single) and FP64 into vin.
__global__ void __launch_bounds__(256) k_scale_df(const double2 *__restrict__ w, const double2 *__restrict__ red,
                                                  double host_scale, float4 *__restrict__ vout,
                                                  double2 *__restrict__ vin, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = red ? sqrt(red->x) : host_scale;
  double inv = s > 0.0 ? 1.0 / s : 0.0;
  double2 a = w[i];
  double2 v = make_double2(a.x * inv, a.y * inv);
  float2 r = split_d(v.x), m = split_d(v.y);
  vout[i] = make_float4(r.x, r.y, m.x, m.y);
  vin[i] = v;
}

struct GmresDev {
  double2 *H;    // [restart][ldh] column-major Hessenberg
  double *cs;    // [restart]
  double2 *sn;   // [restart]
  double2 *g;    // [restart+1]
  double2 *y;    // [restart]
  double2 *h1, *h2;  // [restart+1]
  double2 *red;      // [4]
  double *stat;      // [4] host-visible summary
  int ldh;
};

__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }

__global__ void k_cycle_init(GmresDev d, double beta) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int i = 0; i < d.ldh; ++i) d.g[i] = make_double2(0.0, 0.0);
    d.g[0] = make_double2(beta, 0.0);
  }
}

// Column j of H from the two CGS passes, old rotations, new rotation, g update.
__global__ void k_arnoldi_step(GmresDev d, int j) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 *Hj = d.H + (int64_t)j * d.ldh;
  for (int i = 0; i <= j; ++i) Hj[i] = cadd(d.h1[i], d.h2[i]);
  double hn = sqrt(d.red[0].x);
  Hj[j + 1] = make_double2(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    double c = d.cs[i];
    double2 s = d.sn[i];
    double2 a = Hj[i], b = Hj[i + 1];
    double2 t0 = make_double2(c * a.x, c * a.y);
    t0 = cfma(s, b, t0);
    double2 sc = make_double2(-s.x, s.y);               // -conj(s)
    double2 t1 = cmul(sc, a);
    t1 = make_double2(t1.x + c * b.x, t1.y + c * b.y);
    Hj[i] = t0;
    Hj[i + 1] = t1;
  }
  double2 a = Hj[j], b = Hj[j + 1];
  double aa = cabs_(a), bb = cabs_(b), c;
  double2 s;
  if (bb == 0.0) {
    c = 1.0; s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0; s = make_double2(b.x / bb, -b.y / bb);
  } else {
    double t = hypot(aa, bb);
    c = aa / t;
    double2 ph = make_double2(a.x / aa, a.y / aa);
    s = cmul(ph, make_double2(b.x / t, -b.y / t));
  }
  d.cs[j] = c;
  d.sn[j] = s;
  double2 nj = make_double2(c * a.x, c * a.y);
  Hj[j] = cfma(s, b, nj);
  Hj[j + 1] = make_double2(0.0, 0.0);
  double2 gj = d.g[j];
  double2 sc = make_double2(-s.x, s.y);
  d.g[j + 1] = cmul(sc, gj);
  d.g[j] = make_double2(c * gj.x, c * gj.y);
  d.stat[0] = cabs_(d.g[j + 1]);
  d.stat[1] = hn;
  d.stat[2] = (isfinite(hn) && isfinite(d.stat[0])) ? 0.0 : 1.0;
}

// y = H[0:k,0:k]^{-1} g[0:k] (upper triangular).
__global__ void k_trisolve(GmresDev d, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = d.g[i];
    for (int l = i + 1; l < k; ++l) acc = cfms(d.H[(int64_t)l * d.ldh + i], d.y[l], acc);
    double2 hii = d.H[(int64_t)i * d.ldh + i];
    d.y[i] = cmul(acc, cinv(hii));
  }
}

// ---------------------------------------------------------------- workspace
static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

struct KrylovLayout {
  int64_t n;
  int restart, G, Gdf;
  size_t off_V, off_Z, off_w, off_vin, off_part, off_h1, off_h2, off_red, off_H, off_cs, off_sn, off_g, off_y, off_stat, total;
};

static KrylovLayout krylov_layout(int64_t n, int restart) {
  KrylovLayout L;
  L.n = n; L.restart = restart;
  L.G = (int)((n + DCHUNK - 1) / DCHUNK);
  L.Gdf = (int)((n + DFC - 1) / DFC);
  size_t o = 0, c16 = sizeof(double2);
  L.off_V = o; o += al(c16 * n * (restart + 1));
  L.off_Z = o; o += al(c16 * n * restart);
  L.off_w = o; o += al(c16 * n);
  L.off_vin = o; o += al(c16 * n);
  L.off_part = o; o += al(c16 * (size_t)std::max(L.G, L.Gdf) * (restart + 1));
  L.off_h1 = o; o += al(c16 * (restart + 1));
  L.off_h2 = o; o += al(c16 * (restart + 1));
  L.off_red = o; o += al(c16 * 4);
  L.off_H = o; o += al(c16 * (size_t)(restart + 1) * restart);
  L.off_cs = o; o += al(sizeof(double) * restart);
  L.off_sn = o; o += al(c16 * restart);
  L.off_g = o; o += al(c16 * (restart + 1));
  L.off_y = o; o += al(c16 * restart);
  L.off_stat = o; o += al(sizeof(double) * 4);
  L.total = o;
  return L;
}

size_t krylov_bytes(int64_t n, int restart) { return krylov_layout(n, restart).total; }

// ---------------------------------------------------------------- driver
struct Vec {
  hd_ctx *ctx;
  cudaStream_t st;
  KrylovLayout L;
  char *ws;
  double2 *V() const { return reinterpret_cast<double2 *>(ws + L.off_V); }
  double2 *Z() const { return reinterpret_cast<double2 *>(ws + L.off_Z); }
  double2 *w() const { return reinterpret_cast<double2 *>(ws + L.off_w); }
  double2 *part() const { return reinterpret_cast<double2 *>(ws + L.off_part); }
  double2 *vin() const { return reinterpret_cast<double2 *>(ws + L.off_vin); }
  float4 *Vdf() const { return reinterpret_cast<float4 *>(ws + L.off_V); }

  cudaError_t dots_df(int nk, const double2 *x, double2 *out) {
    tic(ctx, T_ARNOLDI, st);
    k_dots_df<<<L.Gdf, 256, sizeof(float4) * DFC, st>>>(Vdf(), L.n, nk, x, L.n, part(), L.Gdf);
    k_reduce<<<nk, 256, 0, st>>>(part(), L.Gdf, out);
    toc(ctx, T_ARNOLDI, st, 2);
    return cudaGetLastError();
  }
  cudaError_t update_df(int nk, const double2 *coef, double2 *w, double2 *norm_out) {
    tic(ctx, T_ARNOLDI, st);
    size_t sm = sizeof(float4) * nk;
    if (norm_out) {
      k_update_df<true><<<L.G, DT, sm, st>>>(Vdf(), L.n, nk, coef, w, w, L.n, part());
      k_reduce<<<1, 256, 0, st>>>(part(), L.G, norm_out);
    } else {
      k_update_df<false><<<L.G, DT, sm, st>>>(Vdf(), L.n, nk, coef, w, w, L.n, nullptr);
    }
    toc(ctx, T_ARNOLDI, st, norm_out ? 2 : 1);
    return cudaGetLastError();
  }

  cudaError_t dots(const double2 *Vb, int nk, const double2 *x, double2 *out) {
    tic(ctx, T_ARNOLDI, st);
    k_dots<<<L.G, DT, sizeof(double2) * (DT / 32) * nk, st>>>(Vb, L.n, nk, x, L.n, part(), L.G);
    k_reduce<<<nk, 256, 0, st>>>(part(), L.G, out);
    toc(ctx, T_ARNOLDI, st, 2);
    return cudaGetLastError();
  }
  cudaError_t update(const double2 *Vb, int nk, const double2 *coef, double sgn, const double2 *base, double2 *y,
                     double2 *norm_out) {
    tic(ctx, T_ARNOLDI, st);
    size_t sm = sizeof(double2) * nk;
    if (norm_out) {
      k_update<true><<<L.G, DT, sm, st>>>(Vb, L.n, nk, coef, sgn, base, y, L.n, part());
      k_reduce<<<1, 256, 0, st>>>(part(), L.G, norm_out);
    } else {
      k_update<false><<<L.G, DT, sm, st>>>(Vb, L.n, nk, coef, sgn, base, y, L.n, nullptr);
    }
    toc(ctx, T_ARNOLDI, st, norm_out ? 2 : 1);
    return cudaGetLastError();
  }
};

#define KCHK(x)                                   \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

int run_gmres_one(hd_ctx *ctx, const double2 *b, double2 *x, const hd_gmres_opts *o, void *kws, void *scratch,
                  hd_gmres_stats *stats, double *host_stat, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t n = (int64_t)ctx->NX * ctx->NY;
  const int R = o->restart;
  Vec v{ctx, st, krylov_layout(n, R), reinterpret_cast<char *>(kws)};
  GmresDev d;
  char *ws = v.ws;
  d.H = reinterpret_cast<double2 *>(ws + v.L.off_H);
  d.cs = reinterpret_cast<double *>(ws + v.L.off_cs);
  d.sn = reinterpret_cast<double2 *>(ws + v.L.off_sn);
  d.g = reinterpret_cast<double2 *>(ws + v.L.off_g);
  d.y = reinterpret_cast<double2 *>(ws + v.L.off_y);
  d.h1 = reinterpret_cast<double2 *>(ws + v.L.off_h1);
  d.h2 = reinterpret_cast<double2 *>(ws + v.L.off_h2);
  d.red = reinterpret_cast<double2 *>(ws + v.L.off_red);
  d.stat = reinterpret_cast<double *>(ws + v.L.off_stat);
  d.ldh = R + 1;
  const unsigned gs = (unsigned)((n + 255) / 256);
  const bool dsm = o->arnoldi == HD_ARNOLDI_DS;
  if (dsm) KCHK(cudaFuncSetAttribute(k_dots_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float4) * DFC)));

  auto read_red = [&](double *out) -> int {
    KCHK(cudaMemcpyAsync(host_stat, d.red, sizeof(double2), cudaMemcpyDeviceToHost, st));
    KCHK(cudaStreamSynchronize(st));
    *out = host_stat[0];
    return HD_OK;
  };

  // ||b||
  KCHK(v.dots(b, 1, b, d.red));
  double bn2;
  int rc = read_red(&bn2);
  if (rc) return rc;
  const double bnorm = std::sqrt(bn2);
  stats->iters = 0; stats->restarts = 0; stats->converged = 0; stats->status = HD_OK;
  stats->relres_est = 1.0; stats->relres_true = 1.0;
  if (!o->use_x0) KCHK(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
  if (!(bnorm > 0.0)) {
    if (!o->use_x0) {
      stats->converged = 1; stats->relres_est = 0; stats->relres_true = 0;
      return HD_OK;
    }
  }
  int iters = 0, cycles = 0;
  for (;;) {
    // true residual r = b - A x (or b itself for x0 = 0 on the first cycle)
    if (o->use_x0 || cycles > 0) {
      tic(ctx, T_MATVEC, st);
      KCHK(launch_residual(ctx, b, x, v.w(), st));
      toc(ctx, T_MATVEC, st, 1);
    } else {
      KCHK(cudaMemcpyAsync(v.w(), b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    }
    KCHK(v.dots(v.w(), 1, v.w(), d.red));
    double rn2;
    rc = read_red(&rn2);
    if (rc) return rc;
    const double beta = std::sqrt(rn2);
    stats->relres_true = bnorm > 0 ? beta / bnorm : 0.0;
    if (!std::isfinite(beta)) { stats->status = HD_ERR_NUMERIC; return HD_ERR_NUMERIC; }
    if (stats->relres_true <= o->rtol) { stats->converged = 1; break; }
    if (iters >= o->max_iters) break;
    tic(ctx, T_ARNOLDI, st);
    k_cycle_init<<<1, 1, 0, st>>>(d, beta);
    if (dsm) k_scale_df<<<gs, 256, 0, st>>>(v.w(), nullptr, beta, v.Vdf(), v.vin(), n);
    else k_scale<<<gs, 256, 0, st>>>(v.w(), nullptr, beta, v.V(), n);
    toc(ctx, T_ARNOLDI, st, 2);
    int k = 0;
    for (int j = 0; j < R; ++j) {
      double2 *vj = dsm ? v.vin() : v.V() + (int64_t)j * n;
      double2 *zj = v.Z() + (int64_t)j * n;
      rc = run_apply(ctx, vj, zj, scratch, st);
      if (rc) return rc;
      tic(ctx, T_MATVEC, st);
      KCHK(launch_matvec(ctx, zj, v.w(), st));
      toc(ctx, T_MATVEC, st, 1);
      if (dsm) {
        KCHK(v.dots_df(j + 1, v.w(), d.h1));
        KCHK(v.update_df(j + 1, d.h1, v.w(), nullptr));
        KCHK(v.dots_df(j + 1, v.w(), d.h2));
        KCHK(v.update_df(j + 1, d.h2, v.w(), d.red));
      } else {
        KCHK(v.dots(v.V(), j + 1, v.w(), d.h1));
        KCHK(v.update(v.V(), j + 1, d.h1, -1.0, v.w(), v.w(), nullptr));
        KCHK(v.dots(v.V(), j + 1, v.w(), d.h2));
        KCHK(v.update(v.V(), j + 1, d.h2, -1.0, v.w(), v.w(), d.red));
      }
      tic(ctx, T_ARNOLDI, st);
      k_arnoldi_step<<<1, 1, 0, st>>>(d, j);
      if (dsm) k_scale_df<<<gs, 256, 0, st>>>(v.w(), d.red, 0.0, v.Vdf() + (int64_t)(j + 1) * n, v.vin(), n);
      else k_scale<<<gs, 256, 0, st>>>(v.w(), d.red, 0.0, v.V() + (int64_t)(j + 1) * n, n);
      toc(ctx, T_ARNOLDI, st, 2);
      KCHK(cudaGetLastError());
      KCHK(cudaMemcpyAsync(host_stat, d.stat, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
      KCHK(cudaStreamSynchronize(st));
      ++iters;
      k = j + 1;
      if (host_stat[2] != 0.0) { stats->status = HD_ERR_NUMERIC; stats->iters = iters; return HD_ERR_NUMERIC; }
      stats->relres_est = bnorm > 0 ? host_stat[0] / bnorm : 0.0;
      if (stats->relres_est <= o->rtol || host_stat[1] == 0.0 || iters >= o->max_iters) break;
    }
    tic(ctx, T_ARNOLDI, st);
    k_trisolve<<<1, 1, 0, st>>>(d, k);
    toc(ctx, T_ARNOLDI, st, 1);
    KCHK(v.update(v.Z(), k, d.y, 1.0, x, x, nullptr));
    ++cycles;
    collect_timers(ctx);
  }
  stats->iters = iters;
  stats->restarts = cycles;
  stats->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (!stats->converged) stats->status = HD_ERR_NOT_CONVERGED;
  return stats->status;
}

}  // namespace hd
