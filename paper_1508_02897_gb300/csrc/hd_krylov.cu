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
// Several right-hand sides are solved in lockstep (one independent FGMRES per
// right-hand side; every kernel takes the right-hand side as blockIdx.y or .z or
// as a thread index): they share each preconditioner launch, whose factor reads
// are then amortised over the group.  A right-hand side that converges stops
// updating its Hessenberg/solution while the others go on.
//
// Kernels: k_dots (block partial sums of V^H w, w held in registers), k_reduce
// (fixed-order sum of the partials: deterministic), k_update (w = base + sgn V c,
// optionally with block partials of ||w||^2), and one-thread-per-right-hand-side
// kernels for the O(restart) Hessenberg/Givens/triangular work.  The host reads
// 32 bytes per right-hand side and Arnoldi step to decide whether to stop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "hd_internal.cuh"

namespace hd {

constexpr int DT = 256;           // threads per block of the vector kernels
constexpr int DE = 8;             // elements per thread
constexpr int DCHUNK = DT * DE;   // elements per block
constexpr int DFC = 2048;         // elements of w staged per block in k_dots_df (32 KB of shared memory)

// Batched addressing: right-hand side r of a family of vectors starts at
// base + r * ld_r; vector k of a basis at + k * ldv.
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// partial[r][k][blk] = sum over the block's chunk of conj(V_r[k][i]) w_r[i], k < nk.
// With `self`, entry nk is ||w_r||^2; with skip[r] set, the block does nothing.
__global__ void __launch_bounds__(DT) k_dots(const double2 *__restrict__ V, int64_t ldv, int64_t ldvr, int nk0,
                                             const double2 *__restrict__ w_all, int64_t ldw, int64_t n,
                                             double2 *__restrict__ partial_all, int G, int64_t ldp,
                                             const int *__restrict__ skip, int self) {
  extern __shared__ double2 red[];  // [DT/32][nk]
  if (skip && skip[blockIdx.y]) return;
  const int nk = nk0 + self;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double2 *w = w_all + (int64_t)blockIdx.y * ldw;
  const double2 *Vr = V + (int64_t)blockIdx.y * ldvr;
  double2 *partial = partial_all + (int64_t)blockIdx.y * ldp;
  const int64_t base = (int64_t)blockIdx.x * DCHUNK + tid;
  double2 wv[DE];
#pragma unroll
  for (int e = 0; e < DE; ++e) {
    int64_t i = base + (int64_t)DT * e;
    wv[e] = i < n ? w[i] : make_double2(0.0, 0.0);
  }
  for (int k = 0; k < nk; ++k) {
    const double2 *vk = Vr + (int64_t)k * ldv;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < DE; ++e) {
      int64_t i = base + (int64_t)DT * e;
      if (i < n) acc = cfma_conj(k < nk0 ? vk[i] : wv[e], wv[e], acc);
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

// out[r*ldo + k] = sum_b partial[r][k][b] in a fixed order; grid (nk, nrhs).  For a
// skipped right-hand side the output is zeroed (skip_mode 1) or left as it is (2).
__global__ void __launch_bounds__(256) k_reduce(const double2 *__restrict__ partial, int G, int64_t ldp,
                                                double2 *__restrict__ out, int ldo, const int *__restrict__ skip = nullptr,
                                                int skip_mode = 0) {
  __shared__ double2 sm[256];
  const int k = blockIdx.x, tid = threadIdx.x;
  if (skip && skip[blockIdx.y]) {
    if (skip_mode == 1 && tid == 0) out[(int64_t)blockIdx.y * ldo + k] = make_double2(0.0, 0.0);
    return;
  }
  const double2 *p = partial + (int64_t)blockIdx.y * ldp + (int64_t)k * G;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = tid; b < G; b += 256) acc = cadd(acc, p[b]);
  sm[tid] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) sm[tid] = cadd(sm[tid], sm[tid + s]);
    __syncthreads();
  }
  if (tid == 0) out[(int64_t)blockIdx.y * ldo + k] = sm[0];
}

// y_r = base_r + sgn * sum_{k < nk_r} V_r[k] coef_r[k]; optionally normpart[r][blk] =
// block sum of |y_r|^2.  nk_r = nk_per[r] when nk_per is given, else nk.
template <bool NORM>
__global__ void __launch_bounds__(DT) k_update(const double2 *__restrict__ V, int64_t ldv, int64_t ldvr, int nk,
                                               const int *__restrict__ nk_per, const double2 *__restrict__ coef_all,
                                               int ldc, double sgn, const double2 *base_all, double2 *y_all, int64_t ldy,
                                               int64_t n, double2 *__restrict__ normpart_all, int64_t ldp,
                                               const int *__restrict__ skip) {
  extern __shared__ double2 cs[];  // [nk]
  __shared__ double nsm[DT / 32];
  const int tid = threadIdx.x, r = blockIdx.y;
  if (skip && skip[r]) return;
  const int nkr = nk_per ? nk_per[r] : nk;
  const double2 *coef = coef_all + (int64_t)r * ldc;
  const double2 *Vr = V + (int64_t)r * ldvr;
  const double2 *base = base_all + (int64_t)r * ldy;
  double2 *y = y_all + (int64_t)r * ldy;
  for (int k = tid; k < nkr; k += DT) cs[k] = coef[k];
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * DCHUNK + tid;
  double2 acc[DE];
#pragma unroll
  for (int e = 0; e < DE; ++e) acc[e] = make_double2(0.0, 0.0);
  for (int k = 0; k < nkr; ++k) {
    const double2 *vk = Vr + (int64_t)k * ldv;
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
      double2 bv = base[i];
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
      normpart_all[(int64_t)r * ldp + blockIdx.x] = make_double2(s, 0.0);
    }
  }
}

// v_r = w_r * red[4 r + 1].x, the reciprocal norm left there by k_cycle_init /
// k_arnoldi_step (one FP64 division per right-hand side, not per entry); grid (.., nrhs).
__global__ void __launch_bounds__(256) k_scale(const double2 *__restrict__ w_all, int64_t ldw,
                                               const double2 *__restrict__ red, double2 *__restrict__ v_all,
                                               int64_t ldvr, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = blockIdx.y;
  const double inv = red[4 * r + 1].x;
  double2 a = w_all[(int64_t)r * ldw + i];
  v_all[(int64_t)r * ldvr + i] = make_double2(a.x * inv, a.y * inv);
}

// ---------------------------------------------------------------- double-single Arnoldi
// GB300 runs FP64 at 1/61 of its FP32 rate, which makes an FP64 Gram-Schmidt
// ALU-bound.  In this mode the basis V is stored as pairs of floats (hi, lo)
// with hi + lo equal to the FP64 value to about 2^-48, and the dot products
// and updates use double-single arithmetic (Dekker/Knuth error-free products
// and sums on the FP32 pipes), and the conversions between FP64 and float pairs
// move bit fields instead of issuing conversion instructions (ds_split, ds_f2d).
// The FP64 copy of the newest basis vector feeds the preconditioner; the
// residuals, Hessenberg and Givens work stay FP64, the norms are double-single.

// partial[r][k][blk] = sum over the block's DFC elements of conj(V_r[k][i]) w_r[i].
// With `self`, entry nk is ||w_r||^2; with skip[r] set or live[r] clear (a right-hand
// side of a lockstep batch that has stopped), the block does nothing.
__global__ void __launch_bounds__(256) k_dots_df(const float4 *__restrict__ V, int64_t ldv, int64_t ldvr, int nk0,
                                                 const double2 *__restrict__ w_all, int64_t ldw, int64_t n,
                                                 double2 *__restrict__ partial_all, int G, int64_t ldp,
                                                 const int *__restrict__ skip, const int *__restrict__ live, int self) {
  extern __shared__ float4 wsm[];  // [DFC]
  if ((skip && skip[blockIdx.y]) || (live && !live[blockIdx.y])) return;
  const int nk = nk0 + self;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * DFC;
  const int cnt = (int)min((int64_t)DFC, n - base);
  const double2 *w = w_all + (int64_t)blockIdx.y * ldw;
  const float4 *Vr = V + (int64_t)blockIdx.y * ldvr;
  double2 *partial = partial_all + (int64_t)blockIdx.y * ldp;
  for (int i = tid; i < DFC; i += 256) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < cnt) {
      double2 x = w[base + i];
      float2 r = ds_split(x.x), m = ds_split(x.y);
      v = make_float4(r.x, r.y, m.x, m.y);
    }
    wsm[i] = v;
  }
  __syncthreads();
  for (int k = warp; k < nk; k += 8) {
    const float4 *vk = Vr + (int64_t)k * ldv + base;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int i0 = 0; i0 < cnt; i0 += 512) {   // 16 loads of 16 bytes in flight per lane
      float4 vv[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        int i = i0 + u * 32 + lane;
        vv[u] = i < cnt ? (k < nk0 ? vk[i] : wsm[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float4 a = vv[u], b = wsm[i0 + u * 32 + lane];
        ds_mac(rh, rl, a.x, a.y, b.x, b.y);     // re += ar br
        ds_mac(rh, rl, a.z, a.w, b.z, b.w);     // re += ai bi
        ds_mac(ih, il, a.x, a.y, b.z, b.w);     // im += ar bi
        ds_mac(ih, il, -a.z, -a.w, b.x, b.y);   // im -= ai br
        if ((u & 7) == 7) {
          ds_renorm(rh, rl);
          ds_renorm(ih, il);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
      float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
      ds_add(rh, rl, a, b);
      ds_add(ih, il, c, d);
    }
    if (lane == 0) partial[(int64_t)k * G + blockIdx.x] = make_double2(ds_to_d(rh, rl), ds_to_d(ih, il));
  }
}

// v_r = w_r * red[4 r + 1].x written twice: split into V (double-single) and FP64 into vin
// (the normalised first vector of each restart cycle; later ones are stored lazily).
// SCE elements per thread with all loads issued first (one element per thread left too
// few bytes in flight: 2.6 TB/s at 4096^2).
constexpr int SCE = 4;
__global__ void __launch_bounds__(256) k_scale_df(const double2 *__restrict__ w_all, int64_t ldw,
                                                  const double2 *__restrict__ red, float4 *__restrict__ vout_all,
                                                  int64_t ldvr, double2 *__restrict__ vin_all, int64_t n) {
  const int r = blockIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * (256 * SCE) + threadIdx.x;
  const double inv = red[4 * r + 1].x;
  const double2 *w = w_all + (int64_t)r * ldw;
  double2 a[SCE];
#pragma unroll
  for (int u = 0; u < SCE; ++u) {
    const int64_t i = i0 + 256 * u;
    a[u] = i < n ? w[i] : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int u = 0; u < SCE; ++u) {
    const int64_t i = i0 + 256 * u;
    if (i >= n) break;
    const double2 v = make_double2(a[u].x * inv, a[u].y * inv);
    const float2 cr = ds_split(v.x), ci = ds_split(v.y);
    vout_all[(int64_t)r * ldvr + i] = make_float4(cr.x, cr.y, ci.x, ci.y);
    vin_all[(int64_t)r * n + i] = v;
  }
}

// ---------------------------------------------------------------- small per-RHS work
struct GmresDev {
  double2 *H;        // [nrhs][restart][ldh] column-major Hessenberg per right-hand side
  double *cs;        // [nrhs][restart]
  double2 *sn;       // [nrhs][restart]
  double2 *g;        // [nrhs][ldh]
  double2 *y;        // [nrhs][restart]
  double2 *h1, *h2;  // [nrhs][ldh]
  double2 *red;      // [nrhs][4]
  double *stat;      // [nrhs][4] host-visible summary: |g_{j+1}|, h_{j+1,j}, non-finite flag
  int *live;         // [nrhs] 1 while the right-hand side takes Arnoldi steps
  int *kcnt;         // [nrhs] Arnoldi steps of the current cycle
  double *sc;        // [nrhs][ldh] lazy normalisation: basis vector k is stored as v_k / sc_k
  int ldh, restart, nrhs;
  int lazy;          // 1: stored basis vectors carry the scales sc (double-single mode)
};

__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }

// Selective reorthogonalisation (Rutishauser): the second Gram-Schmidt pass runs
// only if the first one cancelled more than a factor 10 of ||w||, i.e.
// ||w - V h|| < ||w|| / 10; h1[nk] holds ||w||^2 and red[4 r] ||w - V h||^2.
__global__ void k_reorth_decide(GmresDev d, int nk, int *skip) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrhs) return;
  const double w2 = d.h1[(int64_t)r * d.ldh + nk].x;
  double w1 = d.red[4 * r].x;
  if (d.lazy) {   // the first pass wrote g (w - V h), g = lazy_gamma(||w||^2)
    const double g = lazy_gamma(w2);
    w1 /= g * g;
  }
  skip[r] = (w1 >= 0.01 * w2) ? 1 : 0;
  d.stat[4 * r + 3] = (w1 >= 0.01 * w2) ? 0.0 : 1.0;   // second pass taken in this step
}

__global__ void k_cycle_init(GmresDev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrhs) return;
  const double beta = sqrt(d.red[4 * r].x);
  d.red[4 * r + 1] = make_double2(beta > 0.0 ? 1.0 / beta : 0.0, 0.0);
  d.sc[(int64_t)r * d.ldh] = 1.0;   // v_0 = r / beta is stored normalised
  if (!d.live[r]) return;
  double2 *g = d.g + (int64_t)r * d.ldh;
  for (int i = 0; i < d.ldh; ++i) g[i] = make_double2(0.0, 0.0);
  g[0] = make_double2(beta, 0.0);
}

// Column j of H from the two CGS passes, old rotations, new rotation, g update.
// Lazy normalisation (double-single mode): the stored vectors are u_k = v_k / sc_k and
// the preconditioner ran on u_j, so w = A M u_j = (A z_j) / sc_j; the first pass returned
// h1_k = u_k^H w and stored g (w - sum_k sc_k^2 h1_k u_k) with g = lazy_gamma(||w||^2),
// the second (if any) h2_k = u_k^H of that and stored y = g (A z_j - sum_k h_kj v_k) / sc_j;
// hence h_kj = sc_j sc_k (h1_k + h2_k / g), h_{j+1,j} = sc_j ||y|| / g and
// sc_{j+1} = 1 / ||y||.
// The column is formed and rotated in registers (each entry computed from h1 and h2 when
// the rotation reaches it, the rotated lower entry carried to the next rotation) and
// stored once: one thread per right-hand side runs this chain, and a store and reload of
// every entry through global memory would set its length.
__global__ void k_arnoldi_step(GmresDev d, int j) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrhs || !d.live[r]) return;
  double2 *Hj = d.H + ((int64_t)r * d.restart + j) * d.ldh;
  const double2 *h1 = d.h1 + (int64_t)r * d.ldh, *h2 = d.h2 + (int64_t)r * d.ldh;
  double *cs = d.cs + (int64_t)r * d.restart;
  double hn = sqrt(d.red[4 * r].x);
  d.red[4 * r + 1] = make_double2(hn > 0.0 ? 1.0 / hn : 0.0, 0.0);   // for k_scale
  double2 *sn = d.sn + (int64_t)r * d.restart;
  double2 *g = d.g + (int64_t)r * d.ldh;
  double *sc = d.sc + (int64_t)r * d.ldh;
  double sj = 1.0, ginv = 1.0;
  if (d.lazy) {
    sj = sc[j];
    ginv = 1.0 / lazy_gamma(h1[j + 1].x);
    sc[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    hn *= sj * ginv;
  }
  // entry i of the new column: h1 + h2, or (lazy) sc_j sc_i (h1 + h2 / g)
  auto col = [&](int i) -> double2 {
    if (!d.lazy) return cadd(h1[i], h2[i]);
    const double f = sj * sc[i];
    return make_double2(f * (h1[i].x + h2[i].x * ginv), f * (h1[i].y + h2[i].y * ginv));
  };
  // the earlier rotations, applied in order to (a, b) = (H_ij, H_{i+1,j})
  double2 a = col(0);
  for (int i = 0; i < j; ++i) {
    const double c = cs[i];
    const double2 s = sn[i];
    const double2 b = col(i + 1);
    double2 t0 = make_double2(c * a.x, c * a.y);
    t0 = cfma(s, b, t0);
    const double2 msc = make_double2(-s.x, s.y);   // -conj(s)
    double2 t1 = cmul(msc, a);
    t1 = make_double2(t1.x + c * b.x, t1.y + c * b.y);
    Hj[i] = t0;
    a = t1;
  }
  // the new rotation zeroes H_{j+1,j} = hn
  const double2 b = make_double2(hn, 0.0);
  const double aa = cabs_(a), bb = cabs_(b);
  double c;
  double2 s;
  if (bb == 0.0) {
    c = 1.0; s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0; s = make_double2(b.x / bb, -b.y / bb);
  } else {
    const double t = hypot(aa, bb);
    c = aa / t;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    s = cmul(ph, make_double2(b.x / t, -b.y / t));
  }
  cs[j] = c;
  sn[j] = s;
  Hj[j] = cfma(s, b, make_double2(c * a.x, c * a.y));
  Hj[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  g[j + 1] = cmul(make_double2(-s.x, s.y), gj);
  g[j] = make_double2(c * gj.x, c * gj.y);
  double *stat = d.stat + 4 * r;
  stat[0] = cabs_(g[j + 1]);
  stat[1] = hn;
  stat[2] = (isfinite(hn) && isfinite(stat[0])) ? 0.0 : 1.0;
}

// y_r = H_r[0:k,0:k]^{-1} g_r[0:k] (upper triangular), k = kcnt[r].
__global__ void k_trisolve(GmresDev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrhs) return;
  const int k = d.kcnt[r];
  const double2 *H = d.H + (int64_t)r * d.restart * d.ldh;
  const double2 *g = d.g + (int64_t)r * d.ldh;
  double2 *y = d.y + (int64_t)r * d.restart;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int l = i + 1; l < k; ++l) acc = cfms(H[(int64_t)l * d.ldh + i], y[l], acc);
    y[i] = cmul(acc, cinv(H[(int64_t)i * d.ldh + i]));
  }
  if (d.lazy) {   // the stored z'_i = M u_i = z_i / sc_i
    const double *sc = d.sc + (int64_t)r * d.ldh;
    for (int i = 0; i < k; ++i) y[i] = make_double2(y[i].x * sc[i], y[i].y * sc[i]);
  }
}

// ---------------------------------------------------------------- workspace
static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

struct KrylovLayout {
  int64_t n;
  int restart, nrhs, G, Gdf, Gmax;
  size_t off_V, off_Z, off_w, off_vin, off_part, off_h1, off_h2, off_red, off_H, off_cs, off_sn, off_g, off_y,
      off_stat, off_live, off_sc, off_ddm, total;
};

static KrylovLayout krylov_layout(int64_t n, int restart, int nrhs) {
  KrylovLayout L;
  L.n = n; L.restart = restart; L.nrhs = nrhs;
  L.G = (int)((n + DCHUNK - 1) / DCHUNK);
  L.Gdf = (int)((n + DFC - 1) / DFC);
  L.Gmax = std::max(L.G, L.Gdf);
  const size_t c16 = sizeof(double2), B = (size_t)nrhs, R = (size_t)restart;
  size_t o = 0;
  L.off_V = o; o += al(c16 * n * (R + 1) * B);
  L.off_Z = o; o += al(c16 * n * R * B);
  L.off_w = o; o += al(c16 * n * B);
  L.off_vin = o; o += al(c16 * n * B);
  L.off_part = o; o += al(c16 * (size_t)L.Gmax * (R + 1) * B);
  L.off_h1 = o; o += al(c16 * (R + 1) * B);
  L.off_h2 = o; o += al(c16 * (R + 1) * B);
  L.off_red = o; o += al(c16 * 4 * B);
  L.off_H = o; o += al(c16 * (R + 1) * R * B);
  L.off_cs = o; o += al(sizeof(double) * R * B);
  L.off_sn = o; o += al(c16 * R * B);
  L.off_g = o; o += al(c16 * (R + 1) * B);
  L.off_y = o; o += al(c16 * R * B);
  L.off_stat = o; o += al(sizeof(double) * 4 * B);
  L.off_live = o; o += al(sizeof(int) * 3 * B);   // live [B], kcnt [B], skip [B]
  L.off_sc = o; o += al(sizeof(double) * (R + 1) * B);
  L.off_ddm = o; o += al(c16 * 2 * n * B);       // multi-step DDM: residual and correction
  L.total = o;
  return L;
}

size_t krylov_bytes(int64_t n, int restart, int nrhs) { return krylov_layout(n, restart, nrhs).total; }

// ---------------------------------------------------------------- driver
#define KCHK(x)                                      \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

struct Krylov {
  hd_ctx *ctx;
  cudaStream_t st;
  KrylovLayout L;
  char *ws;
  int B;
  const int *live = nullptr;   // double-single kernels skip right-hand sides with live[r] == 0
  template <typename T> T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
  double2 *V() const { return at<double2>(L.off_V); }
  float4 *Vdf() const { return at<float4>(L.off_V); }
  double2 *Z() const { return at<double2>(L.off_Z); }
  double2 *w() const { return at<double2>(L.off_w); }
  double2 *vin() const { return at<double2>(L.off_vin); }
  double2 *part() const { return at<double2>(L.off_part); }
  int64_t ldvr() const { return L.n * (L.restart + 1); }
  int64_t ldp() const { return (int64_t)L.Gmax * (L.restart + 1); }

  // out[r*ldo + k] = V_r[k]^H x_r, k < nk (V given with its per-RHS stride); with self,
  // out[r*ldo + nk] = ||x_r||^2; skipped right-hand sides get zeros.
  cudaError_t dots(const double2 *Vb, int64_t vr, int nk, const double2 *x, double2 *out, int ldo,
                   const int *skip = nullptr, int self = 0) {
    tic(ctx, T_ARNOLDI, st);
    k_dots<<<dim3(L.G, B), DT, sizeof(double2) * (DT / 32) * (nk + self), st>>>(Vb, L.n, vr, nk, x, L.n, L.n, part(),
                                                                               L.G, ldp(), skip, self);
    k_reduce<<<dim3(nk + self, B), 256, 0, st>>>(part(), L.G, ldp(), out, ldo, skip, 1);
    toc(ctx, T_ARNOLDI, st, 2);
    return cudaGetLastError();
  }
  // y_r = base_r + sgn V_r c_r; norm_out[4 r] = ||y_r||^2 (left unchanged for skipped ones).
  cudaError_t update(const double2 *Vb, int64_t vr, int nk, const int *nk_per, const double2 *coef, int ldc,
                     double sgn, const double2 *base, double2 *y, double2 *norm_out, const int *skip = nullptr) {
    tic(ctx, T_ARNOLDI, st);
    size_t sm = sizeof(double2) * std::max(nk, 1);
    if (norm_out) {
      k_update<true><<<dim3(L.G, B), DT, sm, st>>>(Vb, L.n, vr, nk, nk_per, coef, ldc, sgn, base, y, L.n, L.n, part(),
                                                   ldp(), skip);
      k_reduce<<<dim3(1, B), 256, 0, st>>>(part(), L.G, ldp(), norm_out, 4, skip, 2);
    } else {
      k_update<false><<<dim3(L.G, B), DT, sm, st>>>(Vb, L.n, vr, nk, nk_per, coef, ldc, sgn, base, y, L.n, L.n,
                                                    nullptr, 0, skip);
    }
    toc(ctx, T_ARNOLDI, st, norm_out ? 2 : 1);
    return cudaGetLastError();
  }
  cudaError_t dots_df(int nk, const double2 *x, double2 *out, int ldo, const int *skip = nullptr, int self = 0) {
    tic(ctx, T_ARNOLDI, st);
    int G = L.Gdf;
    if (nk <= kGsDotsMax) {   // streamed through a shared-memory ring (hd_gs.cu)
      G = gs_items(L.n);
      const cudaError_t e = launch_gs_dots(Vdf(), L.n, ldvr(), nk, x, L.n, L.n, B, part(), ldp(), skip, live, self,
                                           ctx->d_status, st);
      if (e != cudaSuccess) return e;
    } else {
      k_dots_df<<<dim3(L.Gdf, B), 256, sizeof(float4) * DFC, st>>>(Vdf(), L.n, ldvr(), nk, x, L.n, L.n, part(), L.Gdf,
                                                                   ldp(), skip, live, self);
    }
    k_reduce<<<dim3(nk + self, B), 256, 0, st>>>(part(), G, ldp(), out, ldo, skip, 1);
    toc(ctx, T_ARNOLDI, st, 2);
    return cudaGetLastError();
  }
  // y = g (base - V (coef sc^2)) into vin (FP64) and into basis slot nk (float pairs)
  cudaError_t update_df(int nk, const double2 *coef, int ldc, const double *sc, const double2 *base,
                        double2 *norm_out, int scale, const int *skip = nullptr) {
    tic(ctx, T_ARNOLDI, st);
    float4 *vout = Vdf() + (int64_t)nk * L.n;
    const cudaError_t e = launch_gs_update(Vdf(), L.n, ldvr(), nk, coef, ldc, sc, base, vin(), L.n, vout, L.n, B,
                                           norm_out ? part() : nullptr, ldp(), skip, live, scale, ctx->d_status, st);
    if (e != cudaSuccess) return e;
    if (norm_out) k_reduce<<<dim3(1, B), 256, 0, st>>>(part(), gs_items(L.n), ldp(), norm_out, 4, skip, 2);
    toc(ctx, T_ARNOLDI, st, norm_out ? 2 : 1);
    return cudaGetLastError();
  }
};

static int run_gmres_batch_on(hd_ctx *ctx, const double2 *b, double2 *x, int B, const hd_gmres_opts *o, void *kws,
                              void *scratch, hd_gmres_stats *stats, cudaStream_t st);

// With graphs on, the solve runs on a stream of the context (the legacy default
// stream cannot be captured), ordered after and before the caller's stream by events.
int run_gmres_batch(hd_ctx *ctx, const double2 *b, double2 *x, int B, const hd_gmres_opts *o, void *kws,
                    void *scratch, hd_gmres_stats *stats, cudaStream_t st) {
  if (!o->graphs) return run_gmres_batch_on(ctx, b, x, B, o, kws, scratch, stats, st);
  if (!ctx->gstream) {
    KCHK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    KCHK(cudaEventCreateWithFlags(&ctx->gevent, cudaEventDisableTiming));
  }
  KCHK(cudaEventRecord(ctx->gevent, st));
  KCHK(cudaStreamWaitEvent(ctx->gstream, ctx->gevent, 0));
  const int rc = run_gmres_batch_on(ctx, b, x, B, o, kws, scratch, stats, ctx->gstream);
  KCHK(cudaEventRecord(ctx->gevent, ctx->gstream));
  KCHK(cudaStreamWaitEvent(st, ctx->gevent, 0));
  return rc;
}

static int run_gmres_batch_on(hd_ctx *ctx, const double2 *b, double2 *x, int B, const hd_gmres_opts *o, void *kws,
                              void *scratch, hd_gmres_stats *stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t n = (int64_t)ctx->NX * ctx->NY;
  const int R = o->restart;
  Krylov K{ctx, st, krylov_layout(n, R, B), reinterpret_cast<char *>(kws), B};
  GmresDev d;
  d.H = K.at<double2>(K.L.off_H);
  d.cs = K.at<double>(K.L.off_cs);
  d.sn = K.at<double2>(K.L.off_sn);
  d.g = K.at<double2>(K.L.off_g);
  d.y = K.at<double2>(K.L.off_y);
  d.h1 = K.at<double2>(K.L.off_h1);
  d.h2 = K.at<double2>(K.L.off_h2);
  d.red = K.at<double2>(K.L.off_red);
  d.stat = K.at<double>(K.L.off_stat);
  d.live = K.at<int>(K.L.off_live);
  d.sc = K.at<double>(K.L.off_sc);
  K.live = d.live;
  d.kcnt = d.live + B;
  int *skip = d.live + 2 * B;
  const bool sel = o->reorth == 1;
  d.ldh = R + 1; d.restart = R; d.nrhs = B;
  const bool dsm = o->arnoldi == HD_ARNOLDI_DS;
  d.lazy = dsm ? 1 : 0;
  if (dsm) KCHK(cudaFuncSetAttribute(k_dots_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float4) * DFC)));
  const dim3 gs((unsigned)((n + 255) / 256), B);
  const dim3 gsc((unsigned)((n + 256 * SCE - 1) / (256 * SCE)), B);
  const unsigned tb = (unsigned)std::min(B, 256), nb = (unsigned)((B + 255) / 256);

  // host mirror: stat [B][4] doubles | red [B][4] complex | live [B] | kcnt [B]
  const size_t hb = sizeof(double) * 4 * B + sizeof(double2) * 4 * B + 2 * sizeof(int) * B;
  if (ctx->host_buf.size() < hb) ctx->host_buf.resize(hb);
  double *h_stat = reinterpret_cast<double *>(ctx->host_buf.data());
  double2 *h_red = reinterpret_cast<double2 *>(h_stat + 4 * B);
  int *h_live = reinterpret_cast<int *>(h_red + 4 * B);
  int *h_kcnt = h_live + B;

  auto read_red = [&]() -> int {
    KCHK(cudaMemcpyAsync(h_red, d.red, sizeof(double2) * 4 * B, cudaMemcpyDeviceToHost, st));
    KCHK(cudaStreamSynchronize(st));
    return HD_OK;
  };
  auto push_masks = [&]() -> int {
    KCHK(cudaMemcpyAsync(d.live, h_live, sizeof(int) * 2 * B, cudaMemcpyHostToDevice, st));  // live and kcnt are adjacent
    return HD_OK;
  };
  static_assert(sizeof(int) == 4, "int layout");

  // ||b_r||
  KCHK(K.dots(b, n, 1, b, d.red, 4));
  int rc = read_red();
  if (rc) return rc;
  std::vector<double> bnorm(B), rel_est(B, 1.0), rel_true(B, 1.0);
  std::vector<int> iters(B, 0), done(B, 0), conv(B, 0), status(B, HD_OK), passes2(B, 0), vecs2(B, 0);
  for (int r = 0; r < B; ++r) bnorm[r] = std::sqrt(h_red[4 * r].x);
  if (!o->use_x0) KCHK(cudaMemsetAsync(x, 0, sizeof(double2) * n * B, st));
  int cycles = 0;
  for (;;) {
    // true residual r = b - A x (or b itself for x0 = 0 on the first cycle)
    if (o->use_x0 || cycles > 0) {
      tic(ctx, T_MATVEC, st);
      KCHK(launch_residual(ctx, b, x, K.w(), B, st));
      toc(ctx, T_MATVEC, st, 1);
    } else {
      KCHK(cudaMemcpyAsync(K.w(), b, sizeof(double2) * n * B, cudaMemcpyDeviceToDevice, st));
    }
    KCHK(K.dots(K.w(), n, 1, K.w(), d.red, 4));
    rc = read_red();
    if (rc) return rc;
    bool any = false;
    for (int r = 0; r < B; ++r) {
      if (done[r]) { h_live[r] = 0; h_kcnt[r] = 0; continue; }
      const double beta = std::sqrt(h_red[4 * r].x);
      rel_true[r] = bnorm[r] > 0 ? beta / bnorm[r] : 0.0;
      if (!std::isfinite(beta)) { status[r] = HD_ERR_NUMERIC; done[r] = 1; }
      else if (rel_true[r] <= o->rtol) { conv[r] = 1; done[r] = 1; }
      else if (iters[r] >= o->max_iters) { done[r] = 1; }
      h_live[r] = !done[r];
      h_kcnt[r] = 0;
      any = any || !done[r];
    }
    if (!any) break;
    if ((rc = push_masks())) return rc;
    tic(ctx, T_ARNOLDI, st);
    k_cycle_init<<<nb, tb, 0, st>>>(d);
    if (dsm) k_scale_df<<<gsc, 256, 0, st>>>(K.w(), n, d.red, K.Vdf(), K.ldvr(), K.vin(), n);
    else k_scale<<<gs, 256, 0, st>>>(K.w(), n, d.red, K.V(), K.ldvr(), n);
    toc(ctx, T_ARNOLDI, st, 2);
    // One Arnoldi step for every live right-hand side: z_j = M v_j, w = A z_j, CGS2,
    // Hessenberg/Givens update, v_{j+1} = w / ||w||.
    auto enqueue_step = [&](int j) -> int {
      const double2 *vj = dsm ? K.vin() : K.V() + (int64_t)j * n;
      const int64_t vjs = dsm ? n : K.ldvr();
      double2 *zj = K.Z() + (int64_t)j * n;
      const int64_t zs = n * R;
      int rc2 = run_apply_steps(ctx, vj, vjs, zj, zs, B, std::max(1, o->precond_steps), K.at<double2>(K.L.off_ddm),
                                scratch, st);
      if (rc2) return rc2;
      // CGS2: h1 = V^H w, w -= V h1, h2 = V^H w, w -= V h2; with selective
      // reorthogonalisation the second pass is skipped (h2 = 0) unless the first
      // cancelled more than a factor 10 of ||w||.
      const int self = (sel || dsm) ? 1 : 0;   // ||w||^2: the selective rule, the lazy scale
      tic(ctx, T_MATVEC, st);
      KCHK(launch_matvec(ctx, zj, zs, K.w(), n, B, st));
      toc(ctx, T_MATVEC, st, 1);
      if (dsm) {
        // the vector left after each pass goes straight to vin and basis slot j + 1,
        // unnormalised (k_arnoldi_step records its scale)
        KCHK(K.dots_df(j + 1, K.w(), d.h1, R + 1, nullptr, self));
        KCHK(K.update_df(j + 1, d.h1, R + 1, d.sc, K.w(), sel ? d.red : nullptr, 1));
        if (sel) k_reorth_decide<<<nb, tb, 0, st>>>(d, j + 1, skip);
        KCHK(K.dots_df(j + 1, K.vin(), d.h2, R + 1, sel ? skip : nullptr));
        KCHK(K.update_df(j + 1, d.h2, R + 1, d.sc, K.vin(), d.red, 0, sel ? skip : nullptr));
      } else {
        KCHK(K.dots(K.V(), K.ldvr(), j + 1, K.w(), d.h1, R + 1, nullptr, self));
        KCHK(K.update(K.V(), K.ldvr(), j + 1, nullptr, d.h1, R + 1, -1.0, K.w(), K.w(), sel ? d.red : nullptr));
        if (sel) k_reorth_decide<<<nb, tb, 0, st>>>(d, j + 1, skip);
        KCHK(K.dots(K.V(), K.ldvr(), j + 1, K.w(), d.h2, R + 1, sel ? skip : nullptr));
        KCHK(K.update(K.V(), K.ldvr(), j + 1, nullptr, d.h2, R + 1, -1.0, K.w(), K.w(), d.red, sel ? skip : nullptr));
      }
      if (sel) ctx->t_launch[T_ARNOLDI] += 1;
      tic(ctx, T_ARNOLDI, st);
      k_arnoldi_step<<<nb, tb, 0, st>>>(d, j);
      if (!dsm) k_scale<<<gs, 256, 0, st>>>(K.w(), n, d.red, K.V() + (int64_t)(j + 1) * n, K.ldvr(), n);
      toc(ctx, T_ARNOLDI, st, dsm ? 1 : 2);
      KCHK(cudaGetLastError());
      return HD_OK;
    };
    for (int j = 0; j < R; ++j) {
      if (o->graphs) {
        // each step j is captured once per workspace/launch shape and then replayed
        const GraphKey key{kws,          scratch, ctx->factor, B, R,
                           (dsm ? 1 : 0) | (sel ? 2 : 0) | (std::max(1, o->precond_steps) << 2), j, ctx->tune_ct,
                           ctx->tune_ns};
        auto it = ctx->graphs.find(key);
        if (it == ctx->graphs.end()) {
          const bool prof = ctx->profiling;
          int64_t before[T_NCLASS];
          for (int q = 0; q < T_NCLASS; ++q) before[q] = ctx->t_launch[q];
          ctx->profiling = false;   // no event brackets inside a graph
          KCHK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
          const int rc2 = enqueue_step(j);
          cudaGraph_t graph = nullptr;
          const cudaError_t ec = cudaStreamEndCapture(st, &graph);
          ctx->profiling = prof;
          if (rc2) { if (graph) cudaGraphDestroy(graph); return rc2; }
          KCHK(ec);
          GraphEntry ge;
          const cudaError_t ei = cudaGraphInstantiate(&ge.exec, graph, 0);
          cudaGraphDestroy(graph);
          KCHK(ei);
          for (int q = 0; q < T_NCLASS; ++q) {
            ge.kernels[q] = ctx->t_launch[q] - before[q];
            ctx->t_launch[q] = before[q];
          }
          it = ctx->graphs.emplace(key, ge).first;
        }
        tic(ctx, T_OTHER, st);
        KCHK(cudaGraphLaunch(it->second.exec, st));
        toc(ctx, T_OTHER, st, 0);
        for (int q = 0; q < T_NCLASS; ++q) ctx->t_launch[q] += it->second.kernels[q];
      } else {
        if ((rc = enqueue_step(j))) return rc;
      }
      KCHK(cudaMemcpyAsync(h_stat, d.stat, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, st));
      KCHK(cudaStreamSynchronize(st));
      bool alive = false, changed = false;
      for (int r = 0; r < B; ++r) {
        if (!h_live[r]) continue;
        ++iters[r];
        h_kcnt[r] = j + 1;
        const double *sr = h_stat + 4 * r;
        if (!sel || sr[3] != 0.0) { ++passes2[r]; vecs2[r] += j + 1; }
        bool stop = false;
        if (sr[2] != 0.0) { status[r] = HD_ERR_NUMERIC; done[r] = 1; stop = true; }
        rel_est[r] = bnorm[r] > 0 ? sr[0] / bnorm[r] : 0.0;
        if (rel_est[r] <= o->rtol || sr[1] == 0.0 || iters[r] >= o->max_iters) stop = true;
        if (stop) { h_live[r] = 0; changed = true; }
        alive = alive || h_live[r];
      }
      if (!alive) break;
      if (changed && (rc = push_masks())) return rc;
    }
    if ((rc = push_masks())) return rc;   // kcnt for the solution update
    tic(ctx, T_ARNOLDI, st);
    k_trisolve<<<nb, tb, 0, st>>>(d);
    toc(ctx, T_ARNOLDI, st, 1);
    KCHK(K.update(K.Z(), (int64_t)n * R, R, d.kcnt, d.y, R, 1.0, x, x, nullptr));
    ++cycles;
    collect_timers(ctx);
  }
  const double ts = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = HD_OK;
  for (int r = 0; r < B; ++r) {
    hd_gmres_stats &sr = stats[r];
    sr.iters = iters[r];
    sr.restarts = cycles;
    sr.converged = conv[r];
    sr.relres_est = rel_est[r];
    sr.relres_true = rel_true[r];
    sr.t_solve_s = ts;
    sr.second_passes = passes2[r];
    sr.second_pass_vecs = vecs2[r];
    sr.status = status[r] != HD_OK ? status[r] : (conv[r] ? HD_OK : HD_ERR_NOT_CONVERGED);
    if (sr.status == HD_ERR_NUMERIC) worst = HD_ERR_NUMERIC;
    else if (sr.status && !worst) worst = sr.status;
  }
  return worst;
}

}  // namespace hd
