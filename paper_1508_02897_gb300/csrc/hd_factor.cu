// Block-tridiagonal factorisation of every local PML problem (Eq. (pmlij)).
//
// Sec. 3 factorises each local problem once with a direct solver.  Ordering the
// unknowns of a box of width m by grid rows makes the local matrix block
// tridiagonal with tridiagonal diagonal blocks D_j and diagonal coupling blocks
// L_j (row j to row j-1) and U_j (row j to row j+1).  Block LU gives
//     S_0 = D_0,   S_j = D_j - L_j S_{j-1}^{-1} U_{j-1},
// and the solve needs only the S_j^{-1}, which are stored (m x m complex,
// column-major with leading dimension ldm = m rounded up to even, so every
// column starts on a 16-byte boundary: entry (r, c) at c*ldm + r) for every
// row j.
//
// One CTA factorises one box.  Each S_j is inverted in place by Gauss-Jordan
// elimination with partial pivoting done implicitly (rows are never moved: the
// pivot of step k is the largest unpivoted entry of column k).  The elimination
// is blocked by panels of PB columns: the panel is eliminated in shared memory,
// recording for every step its multiplier column and pivot, and every other
// column is then streamed once through registers (one warp per column) while
// the PB recorded steps are applied to it.  If the pivot of step k sits in
// row p_k and q = p^{-1}, the in-place result W satisfies
//     S^{-1}[r][c] = W[p_r][q_c],
// which is how the inverse is written out.
#include "hd_internal.cuh"

namespace hd {

constexpr int FT = 512;        // threads per CTA
constexpr int FWARPS = FT / 32;
constexpr int PB = 16;         // panel width

size_t factor_smem_bytes(int prec, int max_m) {
  size_t cs = prec == HD_C64 ? sizeof(float2) : sizeof(double2);
  return cs * (2 * (size_t)PB * max_m + 2 * PB) + sizeof(int) * 3 * (size_t)max_m;
}

template <typename T> __device__ __forceinline__ auto cabs2(T a) { return a.x * a.x + a.y * a.y; }

template <typename R, int NPL>
__global__ void __launch_bounds__(FT, 1)
k_factor(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const double *__restrict__ k2, int NX,
         double h2, C<R> *__restrict__ factor, C<R> *__restrict__ work, int32_t *status) {
  using T = C<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.x];
  const int m = s.ex, rows = s.ey;
  T *P = reinterpret_cast<T *>(smem_raw);   // [PB][m] panel
  T *F = P + PB * m;                         // [PB][m] multiplier columns
  T *X = F + PB * m;                         // [PB] pivot-row values of the panel
  T *IPV = X + PB;                           // [PB] reciprocal pivots
  int *piv = reinterpret_cast<int *>(IPV + PB);  // [m] pivot row of step k
  int *qinv = piv + m;                           // [m] step at which row r was pivot
  int *done = qinv + m;                          // [m]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double2 *a1c = pool + s.aoff;
  const double2 *ia1f = a1c + m;
  const double2 *a2c = ia1f + m + 1;
  const double2 *ia2f = a2c + rows;
  T *W = work + s.woff;
  T *Fs = factor + s.foff;
  const int ldm = s.ldm;
  const int64_t mm = (int64_t)m * m, slot_elems = (int64_t)m * ldm;
  bool bad = false;

  for (int j = 0; j < rows; ++j) {
    // ---- S_j = D_j - L_j S_{j-1}^{-1} U_{j-1} into W (column-major)
    const T *prev = Fs + (j - 1) * slot_elems;
    const double2 a2 = a2c[j], is = ia2f[j], in = ia2f[j + 1];
    const int gy = s.ey0 + j;
    for (int64_t idx = tid; idx < mm; idx += FT) {
      int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
      T v = mk<T>(0, 0);
      if (r == c) {
        double2 a1 = a1c[r];
        double2 cw = cmul(a2, ia1f[r]), ce = cmul(a2, ia1f[r + 1]);
        double2 cs = cmul(a1, is), cn = cmul(a1, in);
        double2 j12 = cmul(a1, a2);
        double hk = h2 * k2[(int64_t)gy * NX + s.ex0 + r];
        v = mk<T>((R)(-(cw.x + ce.x + cs.x + cn.x) + hk * j12.x), (R)(-(cw.y + ce.y + cs.y + cn.y) + hk * j12.y));
      } else if (r == c + 1) {
        double2 cw = cmul(a2, ia1f[r]);      // row r couples to column r-1 (west)
        v = mk<T>((R)cw.x, (R)cw.y);
      } else if (r + 1 == c) {
        double2 ce = cmul(a2, ia1f[r + 1]);  // row r couples to column r+1 (east)
        v = mk<T>((R)ce.x, (R)ce.y);
      }
      if (j > 0) {
        double2 lr = cmul(a1c[r], is), lc = cmul(a1c[c], is);
        T l_r = mk<T>((R)lr.x, (R)lr.y), l_c = mk<T>((R)lc.x, (R)lc.y);
        v = cfms(cmul(l_r, prev[(int64_t)c * ldm + r]), l_c, v);
      }
      W[idx] = v;
    }
    for (int r = tid; r < m; r += FT) done[r] = 0;
    __syncthreads();

    // ---- Gauss-Jordan inversion of W with implicit partial pivoting
    for (int k0 = 0; k0 < m; k0 += PB) {
      const int nb = min(PB, m - k0);
      for (int idx = tid; idx < nb * m; idx += FT) {
        int t = idx / m, r = idx - t * m;
        P[idx] = W[(int64_t)(k0 + t) * m + r];
      }
      __syncthreads();
      for (int t = 0; t < nb; ++t) {
        const int k = k0 + t;
        if (warp == 0) {
          R best = (R)-1;
          int bi = m;
          for (int r = lane; r < m; r += 32) {
            if (!done[r]) {
              R v = cabs2(P[t * m + r]);
              if (v > best) { best = v; bi = r; }
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            R ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          if (lane == 0) {
            int p = bi < m ? bi : 0;
            T pv = P[t * m + p];
            piv[k] = p;
            qinv[p] = k;
            done[p] = 1;
            if (!(best > (R)0) || !isfinite(best)) {
              bad = true;
              IPV[t] = mk<T>(0, 0);
            } else {
              IPV[t] = cinv(pv);
            }
          }
        }
        __syncthreads();
        const int p = piv[k];
        const T ip = IPV[t];
        for (int r = tid; r < m; r += FT) F[t * m + r] = P[t * m + r];
        for (int tt = tid; tt < nb; tt += FT) X[tt] = tt == t ? ip : cmul(P[tt * m + p], ip);
        __syncthreads();
        for (int idx = tid; idx < nb * m; idx += FT) {
          int tt = idx / m, r = idx - tt * m;
          T nv;
          if (tt == t) {
            nv = r == p ? ip : mk<T>(-(F[t * m + r].x * ip.x - F[t * m + r].y * ip.y),
                                      -(F[t * m + r].x * ip.y + F[t * m + r].y * ip.x));
          } else {
            const T x = X[tt];
            nv = r == p ? x : cfms(F[t * m + r], x, P[idx]);
          }
          P[idx] = nv;
        }
        __syncthreads();
      }
      // write the eliminated panel back
      for (int idx = tid; idx < nb * m; idx += FT) {
        int t = idx / m, r = idx - t * m;
        W[(int64_t)(k0 + t) * m + r] = P[idx];
      }
      // apply the panel's nb steps to every other column, one warp per column
      for (int c = warp; c < m; c += FWARPS) {
        if (c >= k0 && c < k0 + nb) continue;
        T col[NPL];
        T *wc = W + (int64_t)c * m;
#pragma unroll
        for (int e = 0; e < NPL; ++e) {
          int r = lane + 32 * e;
          col[e] = r < m ? wc[r] : mk<T>(0, 0);
        }
        for (int t = 0; t < nb; ++t) {
          const int p = piv[k0 + t];
          const int pe = p >> 5, pl = p & 31;
          T val = col[0];
#pragma unroll
          for (int e = 1; e < NPL; ++e)
            if (pe == e) val = col[e];
          val.x = __shfl_sync(0xffffffffu, val.x, pl);
          val.y = __shfl_sync(0xffffffffu, val.y, pl);
          const T x = cmul(val, IPV[t]);
#pragma unroll
          for (int e = 0; e < NPL; ++e) {
            int r = lane + 32 * e;
            if (r < m) col[e] = r == p ? x : cfms(F[t * m + r], x, col[e]);
          }
        }
#pragma unroll
        for (int e = 0; e < NPL; ++e) {
          int r = lane + 32 * e;
          if (r < m) wc[r] = col[e];
        }
      }
      __syncthreads();
    }

    // ---- write S_j^{-1}[r][c] = W[p_r][q_c] (column-major) as factor row j
    T *slot = Fs + j * slot_elems;
    for (int64_t idx = tid; idx < mm; idx += FT) {
      int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
      slot[(int64_t)c * ldm + r] = W[(int64_t)qinv[c] * m + piv[r]];
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, ST_ZERO_PIVOT);
}

template <typename R, int NPL>
static cudaError_t launch_factor_t(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  size_t smem = factor_smem_bytes(ctx->prec, ctx->max_m);
  cudaError_t e = cudaFuncSetAttribute(k_factor<R, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<R, NPL><<<ctx->nsub, FT, smem, st>>>(ctx->d_subs, ctx->d_lpool, ctx->d_k2, ctx->NX, ctx->h * ctx->h,
                                               reinterpret_cast<C<R> *>(factor), reinterpret_cast<C<R> *>(work),
                                               ctx->d_status);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_factor_r(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  if (ctx->max_m <= 128) return launch_factor_t<R, 4>(ctx, factor, work, st);
  if (ctx->max_m <= 192) return launch_factor_t<R, 6>(ctx, factor, work, st);
  return launch_factor_t<R, 8>(ctx, factor, work, st);
}

int run_factor(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  tic(ctx, T_FACTOR, st);
  cudaError_t e = ctx->prec == HD_C64 ? launch_factor_r<float>(ctx, factor, work, st)
                                      : launch_factor_r<double>(ctx, factor, work, st);
  toc(ctx, T_FACTOR, st, 1);
  if (e != cudaSuccess) return cuda_fail(e, "k_factor launch");
  return HD_OK;
}

}  // namespace hd
