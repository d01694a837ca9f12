// Block-tridiagonal factorisation of every local PML problem (Eq. (pmlij)).
//
// Sec. 3 factorises each local problem once with a direct solver.  Ordering the
// unknowns of a box of width m by grid rows makes the local matrix block
// tridiagonal with tridiagonal diagonal blocks D_j and diagonal coupling blocks
// L_j (row j to row j-1) and U_j (row j to row j+1).  Block LU gives
//     S_0 = D_0,   S_j = D_j - L_j S_{j-1}^{-1} U_{j-1},
// and the solve needs only the S_j^{-1}, which are stored (m x m complex,
// column-major with leading dimension ldm = m rounded up to a multiple of 4, so every
// column starts on a 16-byte boundary: entry (r, c) at c*ldm + r) for every
// row j.  The matrix is complex symmetric, so U_{j-1} = L_j.
//
// One CTA factorises one box.  Each S_j is inverted in place by Gauss-Jordan
// elimination with partial pivoting done implicitly (rows never move: the
// pivot of step k is the largest unpivoted entry of column k), blocked by
// panels of PB columns:
//   1. the panel is eliminated in shared memory, one thread per row;
//   2. with T the product of the panel's PB elementary steps and p_t its pivot
//      rows, the eliminated panel column t equals T e_{p_t}, and T leaves
//      e_i unchanged for every non-pivot row i, so every other column c becomes
//          c' = c with rows p_t zeroed  +  sum_t c[p_t] * panel[:, t],
//      a rank-PB update done as a register-tiled complex GEMM (4 x 4 tiles, the
//      four rows of a tile m/4 apart).
// If the pivot of step k sits in row p_k and q = p^{-1}, the in-place result W
// satisfies S^{-1}[r][c] = W[p_r][q_c], which is how the inverse is written out;
// the same pass builds S_{j+1} from the inverse still in compute precision into
// the second working matrix, so the stored copy may be narrower (FP16 storage
// with FP32 arithmetic) without feeding its rounding back into the recursion.
#include "hd_internal.cuh"

namespace hd {

constexpr int FT = 256;        // threads per CTA (two CTAs, two boxes, share an SM)
constexpr int PB = 16;         // panel width
constexpr int TR = 4, TC = 4;  // GEMM tile of the trailing update (rows x columns)

// Shared memory: panel [PB][m] | B [PB][m] | lS [m] | X [PB] | IPV [PB] | piv, qinv, mark [m] ints
size_t factor_smem_bytes(int prec, int max_m) {
  size_t cs = compute_bytes(prec);
  return cs * (2 * (size_t)PB * max_m + max_m + 2 * PB) + sizeof(int) * 3 * (size_t)max_m + 16;
}

template <typename T> __device__ __forceinline__ auto cabs2(T a) { return a.x * a.x + a.y * a.y; }

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

template <typename R, typename S, bool SYM>
__global__ void __launch_bounds__(FT, 2)
k_factor(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const double *__restrict__ k2, int NX,
         double h2, S *__restrict__ factor, C<R> *__restrict__ work, int32_t *status) {
  using T = C<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.x];
  const int m = s.ex, rows = s.ey;
  T *P = reinterpret_cast<T *>(smem_raw);   // [PB][m] panel (eliminated in place)
  T *Bm = P + PB * m;                        // [PB][m] pivot rows of the other columns
  T *lS = Bm + PB * m;                       // [m] coupling L_j of the current grid row
  T *X = lS + m;                             // [PB] pivot-row values of the panel
  T *IPV = X + PB;                           // [PB] reciprocal pivots
  int *piv = reinterpret_cast<int *>(IPV + PB);  // [m] pivot row of step k
  int *qinv = piv + m;                           // [m] step at which row r was pivot
  int *mark = qinv + m;                          // [m] panel start at which row r became pivot (-1: not yet)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double2 *a1c = pool + s.aoff;
  const double2 *ia1f = a1c + m;
  const double2 *a2c = ia1f + m + 1;
  const double2 *ia2f = a2c + rows;
  T *W = work + s.woff;            // S_j, inverted in place
  T *W2 = W + (int64_t)m * m;      // S_{j+1} under construction
  S *Fs = factor + s.foff;
  const int ldm = s.ldm;
  const int64_t mt16 = (m + 15) / 16;
  const int64_t mm = (int64_t)m * m, slot_elems = SYM ? mt16 * (mt16 + 1) / 2 * 256 : (int64_t)m * ldm;
  bool bad = false;

  // ---- S_0 = D_0
  for (int64_t idx = tid; idx < mm; idx += FT) {
    const int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
    W[idx] = d_entry<T, R>(r, c, 0, a1c, ia1f, a2c, ia2f, k2 + (int64_t)s.ey0 * NX + s.ex0, h2);
  }
  __syncthreads();

  for (int j = 0; j < rows; ++j) {
    for (int r = tid; r < m; r += FT) mark[r] = -1;
    __syncthreads();

    // ---- Gauss-Jordan inversion of W with implicit partial pivoting
    for (int k0 = 0; k0 < m; k0 += PB) {
      const int nb = min(PB, m - k0);
      for (int idx = tid; idx < nb * m; idx += FT) {
        const int t = idx / m, r = idx - t * m;
        P[idx] = W[(int64_t)(k0 + t) * m + r];
      }
      __syncthreads();
      // 1. eliminate the panel, one thread per row
      for (int t = 0; t < nb; ++t) {
        const int k = k0 + t;
        if (warp == 0) {
          R best = (R)-1;
          int bi = m;
          for (int r = lane; r < m; r += 32) {
            if (mark[r] < 0) {
              const R v = cabs2(P[t * m + r]);
              if (v > best) { best = v; bi = r; }
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          const int p = bi < m ? bi : 0;
          T ip = mk<T>(0, 0);
          if (best > (R)0 && isfinite(best)) ip = cinv(P[t * m + p]);
          else if (lane == 0) bad = true;
          // pivot-row values of every panel column after this step (lanes split the columns)
          for (int tt = lane; tt < nb; tt += 32) X[tt] = tt == t ? ip : cmul(P[tt * m + p], ip);
          __syncwarp();
          if (lane == 0) {
            piv[k] = p;
            qinv[p] = k;
            mark[p] = k0;
            IPV[t] = ip;
          }
        }
        __syncthreads();
        const int p = piv[k];
        const T ip = IPV[t];
        for (int r = tid; r < m; r += FT) {
          const T f = P[t * m + r];   // multiplier of row r (column k before the step)
          for (int tt = 0; tt < nb; ++tt) {
            T nv;
            if (r == p) nv = X[tt];
            else if (tt == t) nv = mk<T>(-(f.x * ip.x - f.y * ip.y), -(f.x * ip.y + f.y * ip.x));
            else nv = cfms(f, X[tt], P[tt * m + r]);
            P[tt * m + r] = nv;
          }
        }
        __syncthreads();
      }
      // 2. write the panel back and gather the pivot rows of the other columns
      const int ncol = m - nb;
      for (int idx = tid; idx < nb * m; idx += FT) {
        const int t = idx / m, r = idx - t * m;
        W[(int64_t)(k0 + t) * m + r] = P[idx];
      }
      for (int idx = tid; idx < nb * ncol; idx += FT) {
        const int t = idx / ncol, cc = idx - t * ncol;
        const int c = cc < k0 ? cc : cc + nb;
        Bm[t * m + cc] = W[(int64_t)c * m + piv[k0 + t]];
      }
      __syncthreads();
      // 3. rank-nb update of every other column: C = C(pivot rows zeroed) + panel * Bm.
      //    A thread's TR rows are q apart so that consecutive threads touch consecutive
      //    rows: conflict-free shared-memory reads of the panel, coalesced C accesses.
      const int q = (m + TR - 1) / TR, tcol = (ncol + TC - 1) / TC;
      for (int tile = tid; tile < q * tcol; tile += FT) {
        const int rr = tile % q, c0 = (tile / q) * TC;
        T acc[TR][TC];
#pragma unroll
        for (int b = 0; b < TC; ++b) {
          const int cc = c0 + b;
          const int c = cc < k0 ? cc : cc + nb;
#pragma unroll
          for (int a = 0; a < TR; ++a) {
            const int r = rr + a * q;
            acc[a][b] = (r < m && cc < ncol && mark[r] != k0) ? W[(int64_t)c * m + r] : mk<T>(0, 0);
          }
        }
        for (int t = 0; t < nb; ++t) {
          T pa[TR], bb[TC];
#pragma unroll
          for (int a = 0; a < TR; ++a) pa[a] = rr + a * q < m ? P[t * m + rr + a * q] : mk<T>(0, 0);
#pragma unroll
          for (int b = 0; b < TC; ++b) bb[b] = c0 + b < ncol ? Bm[t * m + c0 + b] : mk<T>(0, 0);
#pragma unroll
          for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) acc[a][b] = cfma(pa[a], bb[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < TC; ++b) {
          const int cc = c0 + b;
          if (cc >= ncol) continue;
          const int c = cc < k0 ? cc : cc + nb;
#pragma unroll
          for (int a = 0; a < TR; ++a)
            if (rr + a * q < m) W[(int64_t)c * m + rr + a * q] = acc[a][b];
        }
      }
      __syncthreads();
    }

    // ---- write S_j^{-1}[r][c] = W[p_r][q_c] (column-major) as factor row j and
    //      build S_{j+1} = D_{j+1} - L_{j+1} S_j^{-1} L_{j+1} from it into W2
    const bool more = j + 1 < rows;
    if (more)
      for (int r = tid; r < m; r += FT) {
        const double2 l = cmul(a1c[r], ia2f[j + 1]);   // south coupling of row j+1
        lS[r] = mk<T>((R)l.x, (R)l.y);
      }
    __syncthreads();
    S *slot = Fs + j * slot_elems;
    const double *k2row = k2 + (int64_t)(s.ey0 + j + 1) * NX + s.ex0;
    if (SYM) {
      // upper 16 x 16 tiles of the exactly symmetric matrix S^{-1}[min(r,c)][max(r,c)],
      // tile (I, J) at J(J+1)/2 + I, entry (r, c) at c*16 + ((r + c) & 15)
      const int mt = (m + 15) / 16;
      const int64_t ntile = (int64_t)mt * (mt + 1) / 2;
      for (int64_t idx = tid; idx < ntile * 256; idx += FT) {
        const int u = (int)(idx >> 8), e = (int)(idx & 255);
        int J = 0;
        while ((J + 1) * (J + 2) / 2 <= u) ++J;
        const int I = u - J * (J + 1) / 2;
        const int cc = e >> 4, rr = ((e & 15) - cc) & 15;
        const int r = I * 16 + rr, c = J * 16 + cc;
        T v = mk<T>(0, 0);
        if (r < m && c < m) v = W[(int64_t)qinv[max(r, c)] * m + piv[min(r, c)]];
        slot[idx] = store_c<S>(v);
      }
      if (more)
        for (int64_t idx = tid; idx < mm; idx += FT) {
          const int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
          const T v = W[(int64_t)qinv[max(r, c)] * m + piv[min(r, c)]];
          W2[idx] = cfms(cmul(lS[r], v), lS[c], d_entry<T, R>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
        }
    } else {
      for (int64_t idx = tid; idx < mm; idx += FT) {
        const int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
        const T v = W[(int64_t)qinv[c] * m + piv[r]];
        slot[(int64_t)c * ldm + r] = store_c<S>(v);
        if (more) W2[idx] = cfms(cmul(lS[r], v), lS[c], d_entry<T, R>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
      }
    }
    __syncthreads();
    T *tmp = W; W = W2; W2 = tmp;
  }
  if (bad) atomicOr(status, ST_ZERO_PIVOT);
}

template <typename R, typename S, bool SYM>
static cudaError_t launch_factor_rs(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  const size_t smem = factor_smem_bytes(ctx->prec, ctx->max_m);
  cudaError_t e = cudaFuncSetAttribute(k_factor<R, S, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<R, S, SYM><<<ctx->nsub, FT, smem, st>>>(ctx->d_subs, ctx->d_lpool, ctx->d_k2, ctx->NX, ctx->h * ctx->h,
                                             reinterpret_cast<S *>(factor), reinterpret_cast<C<R> *>(work),
                                             ctx->d_status);
  return cudaGetLastError();
}

template <typename R, typename S>
static cudaError_t launch_factor_r(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  return ctx->sym ? launch_factor_rs<R, S, true>(ctx, factor, work, st) : launch_factor_rs<R, S, false>(ctx, factor, work, st);
}

int run_factor(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  tic(ctx, T_FACTOR, st);
  cudaError_t e = ctx->prec == HD_C64    ? launch_factor_r<float, float2>(ctx, factor, work, st)
                  : ctx->prec == HD_C64_H ? launch_factor_r<float, __half2>(ctx, factor, work, st)
                                          : launch_factor_r<double, double2>(ctx, factor, work, st);
  toc(ctx, T_FACTOR, st, 1);
  if (e != cudaSuccess) return cuda_fail(e, "k_factor launch");
  return HD_OK;
}

}  // namespace hd
