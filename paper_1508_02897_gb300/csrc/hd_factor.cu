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
//   1. the panel is eliminated with one thread per row (m <= 256 = FT): every
//      thread keeps its row of the panel in registers, publishes it each step
//      into one of two shared buffers (alternating), and the pivot of the next
//      step is found by a block-wide argmax while the current step ends, so a
//      step costs one barrier;
//   2. with T the product of the panel's PB elementary steps and p_t its pivot
//      rows, the eliminated panel column t equals T e_{p_t}, and T leaves
//      e_i unchanged for every non-pivot row i, so every other column c becomes
//          c' = c with rows p_t zeroed  +  sum_t c[p_t] * panel[:, t],
//      a rank-PB update done as a register-tiled complex GEMM (4 x 4 tiles, the
//      four rows of a tile m/4 apart).
// If the pivot of step k sits in row p_k and q = p^{-1}, the in-place result W
// satisfies S^{-1}[r][c] = W[p_r][q_c], which is how the inverse is written out;
// when the stored copy is narrower than the arithmetic (FP16 storage with FP32
// arithmetic) the same pass builds S_{j+1} from the inverse still in compute
// precision into a second working matrix, so storage rounding never feeds back
// into the recursion; otherwise S_{j+1} is built at the start of the next row
// from the stored inverse itself (one working matrix per box, so the working set
// of all resident boxes stays in L2).
#include "hd_internal.cuh"

namespace hd {

constexpr int FT = 256;        // threads per CTA (one box per CTA)
// CTAs per SM the register budget is sized for (two: with three or four resident
// boxes the register cap of 80 or 64 slows the trailing update more than the extra
// boxes hide latency: 528 / 594 / 556 ms for the 4096^2 factorisation).
#ifndef FACTOR_CTAS_F32
#define FACTOR_CTAS_F32 2
#endif
template <typename R> constexpr int factor_ctas() { return sizeof(R) == 4 ? FACTOR_CTAS_F32 : 2; }
constexpr int PB = 16;         // panel width
constexpr int TR = 4, TC = 4;  // GEMM tile of the trailing update (rows x columns)

// Shared memory: panel [PB][m] | B [PB][m] | lS [m] | piv, qinv, mark [m] ints.  During the
// panel elimination B is the second buffer of the published rows.
size_t factor_smem_bytes(int prec, int max_m) {
  size_t cs = compute_bytes(prec);
  return cs * (2 * (size_t)PB * max_m + max_m) + sizeof(int) * 3 * (size_t)max_m + 16;
}

template <typename T> __device__ __forceinline__ auto cabs2(T a) { return a.x * a.x + a.y * a.y; }

// Block-wide argmax of v over the CTA (ties: smaller index); every thread gets the
// result.  sv/si hold one entry per warp; callers alternate two such buffers so a
// fast warp of the next call cannot overwrite what a slow warp still reads.
template <typename R>
__device__ __forceinline__ void block_argmax(R v, int idx, R *sv, int *si, R &best, int &bi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[warp] = v; si[warp] = idx; }
  __syncthreads();
  // second level in every warp: lanes 0..7 take the warps' candidates, three shuffles
  R b2 = lane < FT / 32 ? sv[lane] : (R)-2;
  int i2 = lane < FT / 32 ? si[lane] : 0x7fffffff;
#pragma unroll
  for (int o = (FT / 32) / 2; o > 0; o >>= 1) {
    const R ov = __shfl_xor_sync(0xffffffffu, b2, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i2, o);
    if (ov > b2 || (ov == b2 && oi < i2)) { b2 = ov; i2 = oi; }
  }
  best = __shfl_sync(0xffffffffu, b2, 0);
  bi = __shfl_sync(0xffffffffu, i2, 0);
}

template <typename R, typename S, int LAY>
__global__ void __launch_bounds__(FT, factor_ctas<R>())
k_factor(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const double *__restrict__ k2, int NX,
         double h2, S *__restrict__ factor, C<R> *__restrict__ work, int32_t *status, const int32_t *only) {
  if (only && only[blockIdx.x] == 0) return;   // refactor only the boxes the tensor-core kernel marked
  using T = C<R>;
  constexpr bool SYM = LAY == LAY_SYM, TCL = LAY == LAY_TC || LAY == LAY_TC3;
  constexpr int NPL = LAY == LAY_TC3 ? 4 : 2;   // planes per chunk of the tensor-core layouts
  // S_{j+1} is kept in W2 when the stored copy is narrower than the arithmetic
  constexpr bool KEEP2 = sizeof(S) != sizeof(T) || TCL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.x];
  const int m = s.ex, rows = s.ey;
  T *P = reinterpret_cast<T *>(smem_raw);   // [PB][m] panel (eliminated in place)
  T *Bm = P + PB * m;                        // [PB][m] pivot rows of the other columns
  T *lS = Bm + PB * m;                       // [m] coupling L_j of the current grid row
  int *piv = reinterpret_cast<int *>(lS + m);    // [m] pivot row of step k
  int *qinv = piv + m;                           // [m] step at which row r was pivot
  int *mark = qinv + m;                          // [m] panel start at which row r became pivot (-1: not yet)
  const int tid = threadIdx.x;
  __shared__ R redv[2 * (FT / 32)];
  __shared__ int redi[2 * (FT / 32)];
  const double2 *a1c = pool + s.aoff;
  const double2 *ia1f = a1c + m;
  const double2 *a2c = ia1f + m + 1;
  const double2 *ia2f = a2c + rows;
  T *W = work + s.woff;            // S_j, inverted in place
  T *W2 = W + (int64_t)m * m;      // S_{j+1} under construction
  S *Fs = factor + s.foff;
  const int ldm = s.ldm;
  const int64_t mt16 = (m + 15) / 16;
  const int mp8 = (m + 7) & ~7;
  const int64_t mm = (int64_t)m * m;
  const int64_t slot_elems =
      SYM ? mt16 * (mt16 + 1) / 2 * 256 : (TCL ? (int64_t)(NPL / 2) * mp8 * mp8 : (int64_t)m * ldm);
  bool bad = false;

  // ---- S_0 = D_0
  for (int64_t idx = tid; idx < mm; idx += FT) {
    const int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
    W[idx] = d_entry<T, R>(r, c, 0, a1c, ia1f, a2c, ia2f, k2 + (int64_t)s.ey0 * NX + s.ex0, h2);
  }
  __syncthreads();

  for (int j = 0; j < rows; ++j) {
    if (!KEEP2 && j > 0) {
      // S_j = D_j - L_j S_{j-1}^{-1} L_j from the stored inverse of row j-1
      for (int r = tid; r < m; r += FT) {
        const double2 l = cmul(a1c[r], ia2f[j]);   // south coupling of row j
        lS[r] = mk<T>((R)l.x, (R)l.y);
      }
      __syncthreads();
      const S *prev = Fs + (int64_t)(j - 1) * slot_elems;
      const double *k2row = k2 + (int64_t)(s.ey0 + j) * NX + s.ex0;
      if (SYM) {
        // tile by tile: stored tile (I, J), I <= J, is block (I, J) of S_{j-1}^{-1} and, off the
        // diagonal, the transpose of block (J, I); one FT-thread pass per tile and block,
        // consecutive threads on consecutive rows of W (and of the tile's storage)
        static_assert(FT == 256, "one thread per tile entry");
        const int mt = (m + 15) / 16;
        for (int J = 0, u = 0; J < mt; ++J)
          for (int I = 0; I <= J; ++I, ++u) {
            const S *tile = prev + (int64_t)u * 256;
            {
              const int cc = tid >> 4, rr = ((tid & 15) - cc) & 15;   // storage order
              const int r = 16 * I + rr, c = 16 * J + cc;
              if (r < m && c < m)
                W[(int64_t)c * m + r] = cfms(cmul(lS[r], load_c<T>(tile[tid])), lS[c],
                                             d_band<T, R>(r, c, j, a1c, ia1f, a2c, ia2f, k2row, h2));
            }
            if (I < J) {
              const int rr = tid >> 4, cc = tid & 15;   // W(16J + cc, 16I + rr) = S(16I + rr, 16J + cc)
              const int r = 16 * J + cc, c = 16 * I + rr;
              if (r < m && c < m)
                W[(int64_t)c * m + r] = cfms(cmul(lS[r], load_c<T>(tile[cc * 16 + ((rr + cc) & 15)])), lS[c],
                                             d_band<T, R>(r, c, j, a1c, ia1f, a2c, ia2f, k2row, h2));
            }
          }
      } else {
        for (int64_t idx = tid; idx < mm; idx += FT) {
          const int c = (int)(idx / m), r = (int)(idx - (int64_t)c * m);
          W[idx] = cfms(cmul(lS[r], load_c<T>(prev[(int64_t)c * ldm + r])), lS[c],
                        d_band<T, R>(r, c, j, a1c, ia1f, a2c, ia2f, k2row, h2));
        }
      }
      __syncthreads();
    }
    for (int r = tid; r < m; r += FT) {
      mark[r] = -1;
      qinv[r] = 0;   // stays a valid index even if a breakdown repeats a pivot row
    }
    __syncthreads();

    // ---- Gauss-Jordan inversion of W with implicit partial pivoting
    for (int k0 = 0; k0 < m; k0 += PB) {
      const int nb = min(PB, m - k0);
      for (int idx = tid; idx < nb * m; idx += FT) {
        const int t = idx / m, r = idx - t * m;
        P[idx] = W[(int64_t)(k0 + t) * m + r];
      }
      __syncthreads();
      // 1. eliminate the panel, one thread per row (row r = tid)
      const bool own = tid < m;
      int mymark = own ? mark[tid] : 0;
      T rv[PB];
#pragma unroll
      for (int tt = 0; tt < PB; ++tt) rv[tt] = (own && tt < nb) ? P[tt * m + tid] : mk<T>(0, 0);
      R best;
      int p;
      block_argmax<R>((own && mymark < 0) ? cabs2(rv[0]) : (R)-1, own ? tid : m, redv, redi, best, p);
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        if (t >= nb) break;
        const int k = k0 + t;
        const T *Pin = (t & 1) ? Bm : P;   // rows as they were before this step
        T *Pout = (t & 1) ? P : Bm;
        const bool ok = best > (R)0 && isfinite(best);
        if (p >= m) p = 0;
        T ip;   // reciprocal pivot: one division per warp, broadcast by shuffle
        {
          T inv = mk<T>(0, 0);
          if ((tid & 31) == 0 && ok) {   // one division: 1/|a|^2, then two products
            const T a = Pin[t * m + p];
            const R d = (R)1 / fma_rn(a.x, a.x, mul_rn(a.y, a.y));
            inv = mk<T>(mul_rn(a.x, d), -mul_rn(a.y, d));
          }
          ip = mk<T>(__shfl_sync(0xffffffffu, inv.x, 0), __shfl_sync(0xffffffffu, inv.y, 0));
        }
        if (tid == 0) {
          if (!ok) bad = true;
          piv[k] = p;
          qinv[p] = k;
        }
        if (own) {
          T f = rv[0];   // multiplier of this row (column k before the step)
#pragma unroll
          for (int tt = 1; tt < PB; ++tt)
            if (tt == t) f = rv[tt];
          const T g = cmul(f, ip);
#pragma unroll
          for (int tt = 0; tt < PB; ++tt) {
            if (tt >= nb) break;
            T nv;
            if (tid == p) nv = tt == t ? ip : cmul(Pin[tt * m + p], ip);   // pivot row / pivot
            else if (tt == t) nv = mk<T>(-g.x, -g.y);
            else nv = cfms(g, Pin[tt * m + p], rv[tt]);                   // row - f/pivot * pivot row
            rv[tt] = nv;
            Pout[tt * m + tid] = nv;
          }
          if (tid == p) { mymark = k0; mark[tid] = k0; }
        }
        if (t + 1 < nb) {
          R cand = (R)-1;
#pragma unroll
          for (int tt = 1; tt < PB; ++tt)
            if (tt == t + 1) cand = (own && mymark < 0) ? cabs2(rv[tt]) : (R)-1;
          block_argmax<R>(cand, own ? tid : m, redv + ((t + 1) & 1) * (FT / 32), redi + ((t + 1) & 1) * (FT / 32),
                          best, p);
        }
      }
      __syncthreads();
      if (own)
#pragma unroll
        for (int tt = 0; tt < PB; ++tt)
          if (tt < nb) P[tt * m + tid] = rv[tt];
      __syncthreads();
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

    // ---- write S_j^{-1}[r][c] = W[p_r][q_c] as factor row j and build
    //      S_{j+1} = D_{j+1} - L_{j+1} S_j^{-1} L_{j+1} from it into W2, 16 columns at a
    //      time: column q_c of W is read contiguously and un-permuted into the shared
    //      buffer Q[cc][r] = S_j^{-1}[r][c0 + cc], from which the stored tiles (or
    //      columns) and W2 are written with consecutive threads on consecutive addresses.
    const bool more = KEEP2 && j + 1 < rows;
    if (more)
      for (int r = tid; r < m; r += FT) {
        const double2 l = cmul(a1c[r], ia2f[j + 1]);   // south coupling of row j+1
        lS[r] = mk<T>((R)l.x, (R)l.y);
      }
    S *slot = Fs + j * slot_elems;
    const double *k2row = k2 + (int64_t)(s.ey0 + j + 1) * NX + s.ex0;
    T *Q = P;
    const int mt = (m + 15) / 16;
    for (int J = 0; J < mt; ++J) {
      const int c0 = 16 * J, nc = min(16, m - c0);
      __syncthreads();   // the previous block's reads of Q are done
      for (int idx = tid; idx < nc * m; idx += FT) {
        const int cc = idx / m, i = idx - cc * m;
        Q[cc * m + qinv[i]] = W[(int64_t)qinv[c0 + cc] * m + i];
      }
      __syncthreads();
      if (SYM) {
        // upper 16 x 16 tiles (I, J), I <= J, of the exactly symmetric matrix
        // S^{-1}[min(r,c)][max(r,c)]: tile at J(J+1)/2 + I, entry (r, c) at c*16 + ((r + c) & 15)
        S *tiles = slot + (int64_t)(J * (J + 1) / 2) * 256;
        for (int e2 = tid; e2 < (J + 1) * 256; e2 += FT) {
          const int I = e2 >> 8, e = e2 & 255;
          const int cc = e >> 4, rr = ((e & 15) - cc) & 15;
          const int r = I * 16 + rr, c = c0 + cc;
          T v = mk<T>(0, 0);
          if (r < m && c < m) v = r <= c ? Q[cc * m + r] : Q[(r - c0) * m + c];
          tiles[e2] = store_c<S>(v);
        }
        if (more) {
          // entries (r, c), r <= c, of the block's columns ...
          for (int idx = tid; idx < nc * m; idx += FT) {
            const int cc = idx / m, r = idx - cc * m, c = c0 + cc;
            if (r <= c)
              W2[(int64_t)c * m + r] =
                  cfms(cmul(lS[r], Q[cc * m + r]), lS[c], d_band<T, R>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
          }
          // ... and their mirror images (c, r) below the diagonal
          for (int idx = tid; idx < 16 * m; idx += FT) {
            const int cc = idx & 15, r = idx >> 4, c = c0 + cc;
            if (cc < nc && r < c)
              W2[(int64_t)r * m + c] =
                  cfms(cmul(lS[c], Q[cc * m + r]), lS[r], d_band<T, R>(c, r, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
          }
        }
      } else {
        for (int idx = tid; idx < nc * m; idx += FT) {
          const int cc = idx / m, r = idx - cc * m, c = c0 + cc;
          const T v = Q[cc * m + r];
          if (!TCL) slot[(int64_t)c * ldm + r] = store_c<S>(v);
          if (more) W2[(int64_t)c * m + r] = cfms(cmul(lS[r], v), lS[c], d_band<T, R>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
        }
        if (TCL) {
          // chunks 2J, 2J+1 (8 columns each) of the block, each the real then the imaginary
          // plane [mp8/8 row groups][2 core matrices along K][8 rows][4 columns], TF32
          // (LAY_TC3: then the real and imaginary remainders, also TF32)
          float *F = reinterpret_cast<float *>(slot);
          const int per = 8 * mp8;   // floats of one plane of one chunk
          for (int idx = tid; idx < 2 * NPL * per; idx += FT) {
            const int cp = idx / per, w = idx - cp * per;
            const int ch = 2 * J + cp / NPL, P = cp % NPL;
            if (ch >= mp8 / 8) continue;
            const int g = w >> 6, kk = (w >> 5) & 1, rr = (w >> 2) & 7, c4 = w & 3;
            const int r = 8 * g + rr, c = 8 * ch + 4 * kk + c4;
            float v = 0.f;
            if (r < m && c < m) {
              const T q = Q[(c - c0) * m + r];
              const float x = (float)((P & 1) ? q.y : q.x);
              v = tf32_round(x);
              if (P >= 2) v = tf32_round(x - v);
            }
            F[(int64_t)ch * NPL * per + (int64_t)P * per + w] = v;
          }
        }
      }
    }
    __syncthreads();
    if (KEEP2) { T *tmp = W; W = W2; W2 = tmp; }
  }
  if (bad) atomicOr(status, ST_ZERO_PIVOT);
}

template <typename R, typename S, int LAY>
static cudaError_t launch_factor_rs(hd_ctx *ctx, void *factor, void *work, const int32_t *only, cudaStream_t st) {
  const size_t smem = factor_smem_bytes(ctx->prec, ctx->max_m);
  cudaError_t e = allow_smem(k_factor<R, S, LAY>, smem);
  if (e != cudaSuccess) return e;
  k_factor<R, S, LAY><<<ctx->nsub, FT, smem, st>>>(ctx->d_subs, ctx->d_lpool, ctx->d_k2, ctx->NX, ctx->h * ctx->h,
                                             reinterpret_cast<S *>(factor), reinterpret_cast<C<R> *>(work),
                                             ctx->d_status, only);
  return cudaGetLastError();
}

template <typename R, typename S>
static cudaError_t launch_factor_r(hd_ctx *ctx, void *factor, void *work, const int32_t *only, cudaStream_t st) {
  if (ctx->sym) return launch_factor_rs<R, S, LAY_SYM>(ctx, factor, work, only, st);
  return launch_factor_rs<R, S, LAY_FULL>(ctx, factor, work, only, st);
}

static cudaError_t launch_factor_simt(hd_ctx *ctx, void *factor, void *work, const int32_t *only, cudaStream_t st) {
  return ctx->tc3                 ? launch_factor_rs<float, float2, LAY_TC3>(ctx, factor, work, only, st)
         : ctx->tc               ? launch_factor_rs<float, float2, LAY_TC>(ctx, factor, work, only, st)
         : ctx->prec == HD_C64   ? launch_factor_r<float, float2>(ctx, factor, work, only, st)
         : ctx->prec == HD_C64_H ? launch_factor_r<float, __half2>(ctx, factor, work, only, st)
         : ctx->prec == HD_C64_B ? launch_factor_r<float, __nv_bfloat162>(ctx, factor, work, only, st)
                                 : launch_factor_r<double, double2>(ctx, factor, work, only, st);
}

// The tensor-core kernel where it applies (complex FP32 arithmetic, boxes up to 192
// wide, unless the SIMT kernel was selected), followed by the pivoted SIMT kernel on
// the boxes it marked (a launch whose other CTAs return at once); otherwise the SIMT
// kernel on every box.
int run_factor(hd_ctx *ctx, void *factor, void *work, cudaStream_t st) {
  const bool tcore = ctx->fpath != HD_FACTOR_SIMT && factor_tc_supported(ctx);
  if (ctx->fpath == HD_FACTOR_TCORE && !tcore) {
    set_error("hd_factor_subdomains: the tensor-core factorisation needs complex FP32 factors and boxes at most 192 wide");
    return HD_ERR_INVALID;
  }
  tic(ctx, T_FACTOR, st);
  cudaError_t e = cudaSuccess;
  if (tcore) {
    e = launch_factor_tc(ctx, factor, st);
    if (e == cudaSuccess) e = launch_factor_simt(ctx, factor, work, ctx->d_fflag, st);
  } else {
    e = launch_factor_simt(ctx, factor, work, nullptr, st);
  }
  toc(ctx, T_FACTOR, st, tcore ? 2 : 1);
  if (e != cudaSuccess) return cuda_fail(e, "factorisation launch");
  ctx->last_fpath = tcore ? HD_FACTOR_TCORE : HD_FACTOR_SIMT;
  return HD_OK;
}

}  // namespace hd
