// Preconditioner application, Eq. (ddm0) + Eq. (pc):
//   z = sum_ij E_ij^T A_ij^{-1} X_ij r.
//
// k_subst (one CTA per box) fuses the restriction X_ij r (a gather of the
// owned part of each grid row of the box straight from the global residual)
// with the forward block substitution
//     w_0 = S_0^{-1} rho_0,   w_j = S_j^{-1} (rho_j - L_j w_{j-1}),
// and the back substitution
//     x_last = w_last,        x_j = w_j - S_j^{-1} (U_j x_{j+1}),
// leaving the local solution over the whole box (PML area included) in the
// staging buffer.  Each step is one m x m complex GEMV against a stored
// S_j^{-1}; thread t owns outputs a = t + ST*e and reads column-major entries
// (b, a) for consecutive a, so every factor row is one coalesced stream.
//
// k_gather then forms z cell by cell as a fixed-order sum over the (at most
// 3 x 3, in practice 2 x 2) boxes whose extent covers the cell: deterministic,
// no atomics.
#include "hd_internal.cuh"

namespace hd {

template <typename R, int ST, int NA>
__global__ void __launch_bounds__(ST)
k_subst(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const C<R> *__restrict__ factor,
        const double2 *__restrict__ rg, int NX, C<R> *__restrict__ staging) {
  using T = C<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *vs = reinterpret_cast<T *>(smem_raw);  // [m] right-hand side of the current step
  const SubDev s = subs[blockIdx.x];
  const int m = s.ex, rows = s.ey;
  const int tid = threadIdx.x;
  const double2 *a1c = pool + s.aoff;
  const double2 *a2c = a1c + 2 * m + 1;
  const double2 *ia2f = a2c + rows;
  const T *Fs = factor + s.foff;
  T *stg = staging + s.soff;
  const int64_t mm = (int64_t)m * m;

  T a1[NA], w[NA];
  bool ownx[NA];
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    int a = tid + ST * e;
    int gx = s.ex0 + a;
    ownx[e] = a < m && gx >= s.ox0 && gx < s.ox1;
    double2 t = a < m ? a1c[a] : make_double2(0, 0);
    a1[e] = mk<T>((R)t.x, (R)t.y);
    w[e] = mk<T>(0, 0);
  }

  // ---- forward: restrict + w_j = S_j^{-1}(rho_j - L_j w_{j-1})
  for (int j = 0; j < rows; ++j) {
    const int gy = s.ey0 + j;
    const bool owny = gy >= s.oy0 && gy < s.oy1;
    const double2 isd = ia2f[j];
    const T is = mk<T>((R)isd.x, (R)isd.y);
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      int a = tid + ST * e;
      if (a < m) {
        T rho = mk<T>(0, 0);
        if (owny && ownx[e]) {
          double2 rv = rg[(int64_t)gy * NX + s.ex0 + a];
          rho = mk<T>((R)rv.x, (R)rv.y);
        }
        T v = j > 0 ? cfms(cmul(a1[e], is), w[e], rho) : rho;   // rho - L_j w_{j-1}
        vs[a] = v;
      }
    }
    __syncthreads();
    const T *S = Fs + j * mm;
    T acc[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) acc[e] = mk<T>(0, 0);
    int b = 0;
    for (; b + 8 <= m; b += 8) {
      T mv[8][NA];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int e = 0; e < NA; ++e) {
          int a = tid + ST * e;
          mv[u][e] = a < m ? S[(int64_t)(b + u) * m + a] : mk<T>(0, 0);
        }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        T vb = vs[b + u];
#pragma unroll
        for (int e = 0; e < NA; ++e) acc[e] = cfma(mv[u][e], vb, acc[e]);
      }
    }
    for (; b < m; ++b) {
      T vb = vs[b];
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        int a = tid + ST * e;
        if (a < m) acc[e] = cfma(S[(int64_t)b * m + a], vb, acc[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      int a = tid + ST * e;
      w[e] = acc[e];
      if (a < m) stg[(int64_t)j * m + a] = acc[e];
    }
    __syncthreads();
  }

  // ---- back: x_j = w_j - S_j^{-1}(U_j x_{j+1}); w holds x_{j+1}
  for (int j = rows - 2; j >= 0; --j) {
    const double2 ind = ia2f[j + 1];
    const T in = mk<T>((R)ind.x, (R)ind.y);
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      int a = tid + ST * e;
      if (a < m) vs[a] = cmul(cmul(a1[e], in), w[e]);
    }
    __syncthreads();
    const T *S = Fs + j * mm;
    T acc[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) acc[e] = mk<T>(0, 0);
    int b = 0;
    for (; b + 8 <= m; b += 8) {
      T mv[8][NA];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int e = 0; e < NA; ++e) {
          int a = tid + ST * e;
          mv[u][e] = a < m ? S[(int64_t)(b + u) * m + a] : mk<T>(0, 0);
        }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        T vb = vs[b + u];
#pragma unroll
        for (int e = 0; e < NA; ++e) acc[e] = cfma(mv[u][e], vb, acc[e]);
      }
    }
    for (; b < m; ++b) {
      T vb = vs[b];
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        int a = tid + ST * e;
        if (a < m) acc[e] = cfma(S[(int64_t)b * m + a], vb, acc[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      int a = tid + ST * e;
      if (a < m) {
        T x = csub(stg[(int64_t)j * m + a], acc[e]);
        w[e] = x;
        stg[(int64_t)j * m + a] = x;
      }
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_gather(const SubDev *__restrict__ subs, const AxisDev *__restrict__ axx, const AxisDev *__restrict__ axy,
         const int32_t *__restrict__ nearx, const int32_t *__restrict__ neary, int nbx, int nby,
         const C<R> *__restrict__ staging, double2 *__restrict__ z, int NX) {
  int gx = blockIdx.x * blockDim.x + threadIdx.x;
  int gy = blockIdx.y;
  if (gx >= NX) return;
  const int ix = nearx[gx], iy = neary[gy];
  double2 acc = make_double2(0.0, 0.0);
  for (int jy = max(iy - 1, 0); jy <= min(iy + 1, nby - 1); ++jy) {
    const AxisDev ay = axy[jy];
    if (gy < ay.e0 || gy >= ay.e1) continue;
    for (int jx = max(ix - 1, 0); jx <= min(ix + 1, nbx - 1); ++jx) {
      const AxisDev ax = axx[jx];
      if (gx < ax.e0 || gx >= ax.e1) continue;
      const int64_t base = subs[jy * nbx + jx].soff;
      const int ex = ax.e1 - ax.e0;
      const C<R> v = staging[base + (int64_t)(gy - ay.e0) * ex + (gx - ax.e0)];
      acc.x += (double)v.x;
      acc.y += (double)v.y;
    }
  }
  z[(int64_t)gy * NX + gx] = acc;
}

template <typename R>
static cudaError_t launch_apply_r(hd_ctx *ctx, const double2 *r, double2 *z, void *staging, cudaStream_t st) {
  using T = C<R>;
  const T *F = reinterpret_cast<const T *>(ctx->factor);
  T *S = reinterpret_cast<T *>(staging);
  size_t smem = sizeof(T) * (size_t)ctx->max_m;
  tic(ctx, T_SUBST, st);
  if (ctx->max_m <= 192)
    k_subst<R, 96, 2><<<ctx->nsub, 96, smem, st>>>(ctx->d_subs, ctx->d_lpool, F, r, ctx->NX, S);
  else
    k_subst<R, 128, 2><<<ctx->nsub, 128, smem, st>>>(ctx->d_subs, ctx->d_lpool, F, r, ctx->NX, S);
  toc(ctx, T_SUBST, st, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((ctx->NX + 255) / 256, ctx->NY);
  tic(ctx, T_GATHER, st);
  k_gather<R><<<grid, 256, 0, st>>>(ctx->d_subs, ctx->d_axx, ctx->d_axy, ctx->d_nearx, ctx->d_neary, ctx->nbx,
                                    ctx->nby, S, z, ctx->NX);
  toc(ctx, T_GATHER, st, 1);
  return cudaGetLastError();
}

int run_apply(hd_ctx *ctx, const double2 *r, double2 *z, void *staging, cudaStream_t st) {
  cudaError_t e = ctx->prec == HD_C64 ? launch_apply_r<float>(ctx, r, z, staging, st)
                                      : launch_apply_r<double>(ctx, r, z, staging, st);
  if (e != cudaSuccess) return cuda_fail(e, "preconditioner launch");
  return HD_OK;
}

}  // namespace hd
