// Block-Schur factorisation of every local PML problem (Eq. (pmlij)) on the tensor
// cores, for complex FP32 factors and boxes up to 192 cells wide.
//
// As in hd_factor.cu, each box is block tridiagonal along its grid rows and the
// solve needs S_j^{-1} for S_0 = D_0, S_j = D_j - L_j S_{j-1}^{-1} L_j (L_j diagonal,
// D_j tridiagonal, A complex symmetric).  Here each S_j (m x m) is inverted in place
// by blocked Gauss-Jordan elimination WITHOUT pivoting, in panels of 16 columns.
// On the Schur blocks of these PML problems the diagonal entry is the largest
// remaining one of its column at every step, so the diagonal pivots are the ones
// partial pivoting would pick; every pivot is still checked (below).
//
// The working matrix lives in tensor memory for the whole box (one CTA per SM):
// lane l holds row l, columns [0, NP) the real parts and [NP, 2 NP) the imaginary
// parts of rows 0..127 (NP = m rounded up to 16), and for m > 128 the lanes 0..mb-1
// of columns [2 NP, 2 NP + NB) and [2 NP + NB, 2 NP + 2 NB) hold the bottom-right
// block (rows and columns 128..m-1, mb = m - 128, NB = mb rounded up to 16).  The
// bottom-left block is not stored: Gauss-Jordan on a symmetric matrix keeps the
// eliminated block and the Schur complement symmetric and the two off-diagonal
// blocks negative transposes of each other, so W[r][c] for r >= 128 > c is +-W[c][r]
// (+ while both indices are still unprocessed, which is the only case read).
//
// Eliminating panel K (columns k0 .. k0+w-1) with C = W[:, K], P = C_K^{-1} (the
// w x w diagonal block inverted by the SIMT threads), X = C - E_K and
// Y^T = Z P (Z = C with already eliminated rows negated and rows K replaced by the
// identity; by the symmetry above this is P times the row panel) is one update
//     W <- W with columns K set to E_K,  then  W <- W - X Y,
// which gives all four parts of the in-place Gauss-Jordan step at once (pivot
// block P, row panel P W_KJ, column panel -W_IK P, trailing W_IJ - W_IK P W_KJ).
// W - X Y is a rank-16 complex update accumulated straight into the resident
// matrix by tcgen05.mma kind::f16: every real operand is split into three BF16
// pieces (x = h + m + l exactly to 2^-25 |x|, rounded to nearest), and the six
// products h h, h m, m h, h l, m m, l h of each real product give FP32-grade
// products (the neglected terms are below 2^-25); with FP32 accumulation in tensor
// memory the update matches FP32 arithmetic.  The complex product takes the four
// real products Xr Yr, Xi Yi, Xr Yi, Xi Yr, each accumulated into its real or
// imaginary plane with the sign stored in the operands (A = -Xr, -Xi; B = Yr, Yi,
// -Yi).  One panel is 24 MMAs for rows 0..127 (N = NP) and 24 for the bottom-right
// block (M = 128 rows starting at operand row 128, N = NB).
//
// Pivot check: within each diagonal block every pivot is compared with the other
// unprocessed entries of its column (and, for the first column of the panel, with
// all unprocessed rows below the panel); a pivot smaller than pivot_ratio times the
// largest of them, or a non-finite one, marks the box, and hd_factor_subdomains
// refactors marked boxes with the partially pivoted SIMT kernel right after this one.
//
// After the last panel, S_j^{-1} is read out of tensor memory once: written to the
// factor storage (full column-major, upper 16 x 16 tiles or TF32 planes; complex
// FP32 or FP16) and turned in place into S_{j+1} = D_{j+1} - L S_j^{-1} L, so the
// recursion runs on the FP32 values and storage rounding never feeds back.
#include <cuda_bf16.h>

#include "hd_internal.cuh"
#include "hd_tc.cuh"

namespace hd {

namespace {

constexpr int FX_THREADS = 256;
constexpr int FX_MAXM = 192;     // 2 NP + 2 NB <= 512 tensor-memory columns
constexpr int FX_KP = 16;        // panel width = K of one kind::f16 MMA
constexpr int FX_ROWS = 192;     // rows of the B operand tiles and of the panel copy
constexpr int FX_AROWS = 256;    // rows of the A operand tiles (the bottom MMA reads rows 128..255)
constexpr uint32_t FX_ATILE = FX_AROWS * 32;   // bytes of one A tile: 16 BF16 per row
constexpr uint32_t FX_BTILE = FX_ROWS * 32;
constexpr int FX_NA = 6, FX_NBT = 9;           // A: -Xr, -Xi; B: Yr, Yi, -Yi; three pieces each
constexpr uint32_t FX_TMEM_COLS = 512;
constexpr int CLD = 17;          // row stride (entries) of the panel copy: conflict-free rows and columns

constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + (size_t)FX_NA * FX_ATILE;
constexpr size_t kOffC = kOffB + (size_t)FX_NBT * FX_BTILE;
constexpr size_t kOffG = kOffC + sizeof(float2) * FX_ROWS * CLD;
constexpr size_t kOffL = kOffG + sizeof(float2) * 2 * FX_KP * FX_KP;
constexpr size_t kOffM = kOffL + sizeof(float2) * FX_ROWS;
constexpr size_t kSmem = kOffM + 32;

// x = h + m + l with BF16 pieces rounded to nearest (each remainder is exact in FP32).
__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r1 = __fsub_rn(x, __bfloat162float(bh));
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = __fsub_rn(r1, __bfloat162float(bm));
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

// Row r of an operand tile (16 BF16 values) in the no-swizzle K-major layout: 8-row
// groups 256 bytes apart (SBO), the two 8-column core matrices 128 bytes apart (LBO).
__device__ __forceinline__ void put_row(unsigned char *tile, int r, const uint16_t *v) {
  unsigned char *p = tile + (r >> 3) * 256 + (r & 7) * 16;
  uint4 a, b;
  a.x = v[0] | ((uint32_t)v[1] << 16); a.y = v[2] | ((uint32_t)v[3] << 16);
  a.z = v[4] | ((uint32_t)v[5] << 16); a.w = v[6] | ((uint32_t)v[7] << 16);
  b.x = v[8] | ((uint32_t)v[9] << 16); b.y = v[10] | ((uint32_t)v[11] << 16);
  b.z = v[12] | ((uint32_t)v[13] << 16); b.w = v[14] | ((uint32_t)v[15] << 16);
  *reinterpret_cast<uint4 *>(p) = a;
  *reinterpret_cast<uint4 *>(p + 128) = b;
}

// Splits 16 values and writes the three pieces as row r of tiles t, t+1, t+2.
__device__ __forceinline__ void put_split(unsigned char *tiles, uint32_t tile_bytes, int t, int r, const float *v) {
  uint16_t h[16], m[16], l[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) split3(v[i], h[i], m[i], l[i]);
  put_row(tiles + (size_t)t * tile_bytes, r, h);
  put_row(tiles + (size_t)(t + 1) * tile_bytes, r, m);
  put_row(tiles + (size_t)(t + 2) * tile_bytes, r, l);
}

__device__ __forceinline__ float cabs2f(float2 a) { return a.x * a.x + a.y * a.y; }

// Stored entry (r, c) of S_j^{-1} in the full or tensor-core layouts (zero outside m x m).
template <typename S, int LAY>
__device__ __forceinline__ void emit(S *slot, int r, int c, float2 v, int m, int ldm, int mp8) {
  if (LAY == LAY_FULL) {
    if (r < m && c < m) slot[(int64_t)c * ldm + r] = store_c<S>(v);
  } else {   // LAY_TC: chunk c/8, real then imaginary plane [mp8/8][2][8][4], TF32
    if (r >= mp8 || c >= mp8) return;
    if (r >= m || c >= m) v = make_float2(0.f, 0.f);
    float *F = reinterpret_cast<float *>(slot);
    const int per = 8 * mp8;
    const int64_t o = (int64_t)(c >> 3) * 2 * per + (r >> 3) * 64 + ((c >> 2) & 1) * 32 + (r & 7) * 4 + (c & 3);
    F[o] = tf32_round(v.x);
    F[o + per] = tf32_round(v.y);
  }
}

}  // namespace

size_t factor_tc_smem_bytes() { return kSmem; }

template <typename S, int LAY>
__global__ void __launch_bounds__(FX_THREADS, 1)
k_factor_tc(const SubDev *__restrict__ subs, int nsub, const double2 *__restrict__ pool, const double *__restrict__ k2,
            int NX, double h2, S *__restrict__ factor, float tau2, int32_t *__restrict__ flags, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *At = smem_raw + kOffA;
  unsigned char *Bt = smem_raw + kOffB;
  float2 *Cs = reinterpret_cast<float2 *>(smem_raw + kOffC);   // [FX_ROWS][CLD] panel columns
  float2 *G = reinterpret_cast<float2 *>(smem_raw + kOffG);    // [2][16][16] pivot block
  float2 *lS = reinterpret_cast<float2 *>(smem_raw + kOffL);   // [FX_ROWS] coupling of the next row
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + kOffM);
  uint32_t *tholder = reinterpret_cast<uint32_t *>(mbar + 1);
  volatile int *sflag = reinterpret_cast<volatile int *>(tholder + 1);
  volatile int *abort_flag = sflag + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::bar_init(mbar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(tholder)),
                 "r"(FX_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tholder;
  // this warp's lane quarter in tensor memory
  const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  uint32_t nphase = 0;
  bool alive = true;

  for (int box = blockIdx.x; box < nsub && alive; box += gridDim.x) {
    const SubDev s = subs[box];
    const int m = s.ex, rows = s.ey;
    const int NP = (m + 15) & ~15;
    const int mb = m > 128 ? m - 128 : 0;
    const int NB = (mb + 15) & ~15;
    const int mt = NP / 16, mp8 = (m + 7) & ~7;
    const double2 *a1c = pool + s.aoff;
    const double2 *ia1f = a1c + m;
    const double2 *a2c = ia1f + m + 1;
    const double2 *ia2f = a2c + rows;
    S *Fs = factor + s.foff;
    const int64_t slot_elems = LAY == LAY_SYM ? (int64_t)mt * (mt + 1) / 2 * 256
                                              : (LAY == LAY_TC ? (int64_t)mp8 * mp8 : (int64_t)m * s.ldm);
    const uint32_t idesc_top = tc::idesc_bf16(128, NP);
    const uint32_t idesc_bot = tc::idesc_bf16(128, NB > 0 ? NB : 16);

    // operand tiles and the panel copy start at zero: rows >= m are never written
    for (int i = tid; i < (int)(kOffG / 16); i += FX_THREADS)
      reinterpret_cast<uint4 *>(smem_raw)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) *sflag = 0;

    // ---- S_0 = D_0 into tensor memory
    {
      const double *k2row = k2 + (int64_t)s.ey0 * NX + s.ex0;
      if (warp < 4) {
        const int r = tid;
        for (int cc = 0; cc < NP; cc += 16) {
          float re[16], im[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = cc + i;
            const float2 v = (r < m && c < m) ? d_band<float2, float>(r, c, 0, a1c, ia1f, a2c, ia2f, k2row, h2)
                                              : make_float2(0.f, 0.f);
            re[i] = v.x;
            im[i] = v.y;
          }
          tc::tmem_st16(tq + cc, re);
          tc::tmem_st16(tq + NP + cc, im);
        }
      } else if (warp < 6 && mb > 0) {
        const int r = 128 + tid - 128;   // bottom rows: lane tid - 128 of quarters 0 and 1
        for (int cc = 0; cc < NB; cc += 16) {
          float re[16], im[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = 128 + cc + i;
            const float2 v = (r < m && c < m) ? d_band<float2, float>(r, c, 0, a1c, ia1f, a2c, ia2f, k2row, h2)
                                              : make_float2(0.f, 0.f);
            re[i] = v.x;
            im[i] = v.y;
          }
          tc::tmem_st16(tq + 2 * NP + cc, re);
          tc::tmem_st16(tq + 2 * NP + NB + cc, im);
        }
      }
      tc::tmem_wait_st();
    }

    for (int j = 0; j < rows && alive; ++j) {
      const bool more = j + 1 < rows;
      __syncthreads();   // the previous row's write-out has finished reading lS
      // coupling of the next grid row (used after the last panel)
      if (more)
        for (int r = tid; r < FX_ROWS; r += FX_THREADS) {
          float2 l = make_float2(0.f, 0.f);
          if (r < m) {
            const double2 ld = cmul(a1c[r], ia2f[j + 1]);
            l = make_float2((float)ld.x, (float)ld.y);
          }
          lS[r] = l;
        }

      for (int k0 = 0; k0 < m; k0 += FX_KP) {
        const int w = min(FX_KP, m - k0);
        // ---- A. copy the panel columns C = W[:, K] into shared memory
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (warp < 4) {
          float re[16], im[16];
          tc::tmem_ld16(tq + k0, re);
          tc::tmem_ld16(tq + NP + k0, im);
#pragma unroll
          for (int i = 0; i < 16; ++i) Cs[tid * CLD + i] = make_float2(re[i], im[i]);
        } else if (mb > 0) {
          if (k0 >= 128) {
            if (warp < 6) {   // bottom rows from the bottom-right block
              const int rb = tid - 128;
              float re[16], im[16];
              tc::tmem_ld16(tq + 2 * NP + (k0 - 128), re);
              tc::tmem_ld16(tq + 2 * NP + NB + (k0 - 128), im);
#pragma unroll
              for (int i = 0; i < 16; ++i) Cs[(128 + rb) * CLD + i] = make_float2(re[i], im[i]);
            }
          } else if (warp - 4 == (k0 >> 5)) {
            // bottom rows of panel columns k < 128: W[128 + c'][k] = W[k][128 + c'], held by lane k
            const int row = 32 * (warp - 4) + lane;
            const bool mine = row >= k0 && row < k0 + FX_KP;
            for (int cc = 0; cc < 64; cc += 16) {
              float re[16], im[16];
              if (cc < NB) {
                tc::tmem_ld16(tq + 128 + cc, re);
                tc::tmem_ld16(tq + NP + 128 + cc, im);
              }
              if (mine)
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const int cp = cc + i;
                  Cs[(128 + cp) * CLD + (row - k0)] = cp < mb ? make_float2(re[i], im[i]) : make_float2(0.f, 0.f);
                }
            }
          }
        }
        __syncthreads();

        // ---- B. P = C_K^{-1} (w x w) by Gauss-Jordan without pivoting, with the pivot check
        {
          const int i = tid >> 4, jj = tid & 15;
          G[tid] = (i < w && jj < w) ? Cs[(k0 + i) * CLD + jj] : make_float2(i == jj ? 1.f : 0.f, 0.f);
          if (warp == 7) {
            // first pivot against every unprocessed row below the panel
            float mx = 0.f;
            for (int r = k0 + w + lane; r < m; r += 32) mx = fmaxf(mx, cabs2f(Cs[r * CLD]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const float p2 = cabs2f(Cs[k0 * CLD]);
            if (lane == 0 && !(p2 >= tau2 * mx)) *sflag = 1;
          }
          __syncthreads();
          for (int k = 0; k < w; ++k) {
            const float2 *src = G + (k & 1) * 256;
            float2 *dst = G + ((k + 1) & 1) * 256;
            const float2 piv = src[k * 16 + k];
            const float2 ip = cinv(piv);
            if (tid == 0) {
              float mx = 0.f;
              for (int q = k + 1; q < w; ++q) mx = fmaxf(mx, cabs2f(src[q * 16 + k]));
              const float p2 = cabs2f(piv);
              if (!(p2 >= tau2 * mx) || !(p2 > 0.f) || !isfinite(p2)) *sflag = 1;
            }
            const float2 aik = src[i * 16 + k], akj = src[k * 16 + jj], aij = src[tid];
            float2 v;
            if (i == k) v = jj == k ? ip : cmul(akj, ip);
            else if (jj == k) { v = cmul(aik, ip); v.x = -v.x; v.y = -v.y; }
            else v = cfms(aik, cmul(akj, ip), aij);
            dst[tid] = v;
            __syncthreads();
          }
        }
        const float2 *Pm = G + (w & 1) * 256;   // P[i][kk] at Pm[i * 16 + kk]

        // ---- C. operands: A = -X (X = C outside rows K, zero on rows K) and B = Y^T = Z P,
        //         three BF16 pieces each; Y^T also replaces C in the panel copy
        if (tid < FX_ROWS && tid < m) {
          const int r = tid, kr = r - k0;
          const bool inK = kr >= 0 && kr < w;
          float2 c[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) c[i] = Cs[r * CLD + i];
          float vr[16], vi[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            vr[i] = inK ? 0.f : -c[i].x;
            vi[i] = inK ? 0.f : -c[i].y;
          }
          put_split(At, FX_ATILE, 0, r, vr);
          put_split(At, FX_ATILE, 3, r, vi);
          float2 y[16];
          if (inK) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
              float2 p = make_float2(0.f, 0.f);
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (q == kr) p = Pm[q * 16 + kk];
              y[kk] = (kk < w) ? p : make_float2(0.f, 0.f);
            }
          } else {
            const float zs = r < k0 ? -1.f : 1.f;
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
              float2 acc = make_float2(0.f, 0.f);
              if (kk < w) {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                  if (q < w) acc = cfma(c[q], Pm[q * 16 + kk], acc);
              }
              y[kk] = make_float2(zs * acc.x, zs * acc.y);
            }
          }
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            vr[kk] = y[kk].x;
            vi[kk] = y[kk].y;
            Cs[r * CLD + kk] = y[kk];
          }
          put_split(Bt, FX_BTILE, 0, r, vr);
          put_split(Bt, FX_BTILE, 3, r, vi);
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) vi[kk] = -vi[kk];
          put_split(Bt, FX_BTILE, 6, r, vi);
        }
        __syncthreads();
        // rows K take their new values directly, W[k][:] = Y[k - k0][:] (P on the diagonal
        // block, P W_KJ elsewhere: no cancellation), and every other row gets zero in the
        // columns K, which the update below fills with -C P.  Tensor-memory stores are
        // warp-collective, so the warp holding rows K rewrites whole rows: its other lanes
        // store back what they hold (zero in the columns K).
        {
          const bool kwarp_top = warp < 4 && (k0 >> 5) == warp && k0 < 128;
          const bool kwarp_bot = warp >= 4 && warp < 6 && k0 >= 128 && ((k0 - 128) >> 5) == warp - 4;
          const bool zwarp = (warp < 4) || (warp < 6 && k0 >= 128);
          if (kwarp_top || kwarp_bot) {
            const int kr = tid - k0;   // top: row tid; bottom: row 128 + (tid - 128) = tid
            const bool inK = kr >= 0 && kr < w;
            const int ncol = kwarp_top ? NP : NB, cb = kwarp_top ? 0 : 128, kc = k0 - cb;
            const uint32_t tre = kwarp_top ? tq : tq + 2 * NP, tim = kwarp_top ? tq + NP : tq + 2 * NP + NB;
            for (int cc = 0; cc < ncol; cc += 16) {
              float re[16], im[16];
              tc::tmem_ld16(tre + cc, re);
              tc::tmem_ld16(tim + cc, im);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                if (inK) {
                  const float2 v = Cs[(cb + cc + i) * CLD + kr];
                  re[i] = v.x;
                  im[i] = v.y;
                } else if (cc == kc) {
                  re[i] = 0.f;
                  im[i] = 0.f;
                }
              }
              tc::tmem_st16(tre + cc, re);
              tc::tmem_st16(tim + cc, im);
            }
          } else if (zwarp) {
            const float z[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const uint32_t base = warp < 4 ? tq + k0 : tq + 2 * NP + (k0 - 128);
            const uint32_t off = warp < 4 ? NP : NB;
            tc::tmem_st16(base, z);
            tc::tmem_st16(base + off, z);
          }
        }
        tc::tmem_wait_st();
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();

        // ---- D. W -= X Y on the tensor cores (one thread issues), then wait
        if (tid == 0) {
          tc::fence_after();
          const uint32_t a0 = tc::su32(At), b0 = tc::su32(Bt);
          for (int part = 0; part < (mb > 0 ? 2 : 1); ++part) {
            const uint32_t dr = tmem + (part ? 2 * NP : 0), di = tmem + (part ? 2 * NP + NB : NP);
            const uint32_t ro = part ? 16 * 256 : 0;   // operand row 128: 16 groups of 8 rows
            const uint32_t id = part ? idesc_bot : idesc_top;
#pragma unroll
            for (int pq = 0; pq < 6; ++pq) {
              // piece pairs (p, q) with p + q <= 2: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
              const int p = pq == 2 ? 1 : (pq == 4 ? 1 : (pq == 5 ? 2 : 0));
              const int q = pq == 1 ? 1 : (pq == 3 ? 2 : (pq == 4 ? 1 : 0));
              const uint32_t axr = a0 + (uint32_t)p * FX_ATILE + ro, axi = a0 + (uint32_t)(3 + p) * FX_ATILE + ro;
              const uint32_t byr = b0 + (uint32_t)q * FX_BTILE + ro, byi = b0 + (uint32_t)(3 + q) * FX_BTILE + ro;
              const uint32_t byn = b0 + (uint32_t)(6 + q) * FX_BTILE + ro;
              tc::mma_bf16(dr, tc::mdesc(axr, 128, 256), tc::mdesc(byr, 128, 256), id, 1u);   // -Xr Yr
              tc::mma_bf16(dr, tc::mdesc(axi, 128, 256), tc::mdesc(byn, 128, 256), id, 1u);   // +Xi Yi
              tc::mma_bf16(di, tc::mdesc(axr, 128, 256), tc::mdesc(byi, 128, 256), id, 1u);   // -Xr Yi
              tc::mma_bf16(di, tc::mdesc(axi, 128, 256), tc::mdesc(byr, 128, 256), id, 1u);   // -Xi Yr
            }
          }
          tc::mma_commit(mbar);
        }
        const bool ok = tc::bar_wait(mbar, nphase & 1u, abort_flag);
        ++nphase;
        tc::fence_after();
        if (__syncthreads_or(!ok)) {
          if (tid == 0) {
            *abort_flag = 1;
            atomicOr(status, ST_TIMEOUT);
          }
          alive = false;
          break;
        }
      }
      if (!alive) break;

      // ---- write S_j^{-1} out and turn it into S_{j+1} = D_{j+1} - L S_j^{-1} L in place
      S *slot = Fs + (int64_t)j * slot_elems;
      const double *k2row = k2 + (int64_t)(s.ey0 + j + 1) * NX + s.ex0;
      const int ldm = s.ldm;
      if (warp < 4 || (warp < 6 && mb > 0)) {
        const bool top = warp < 4;
        const int r = top ? tid : tid;   // bottom rows: 128 + (tid - 128)
        const int ncol = top ? NP : NB;
        const int cbase = top ? 0 : 128;
        const uint32_t tre = top ? tq : tq + 2 * NP, tim = top ? tq + NP : tq + 2 * NP + NB;
        const int I = r >> 4, rr = r & 15;
        for (int cc = 0; cc < ncol; cc += 16) {
          float re[16], im[16];
          tc::tmem_ld16(tre + cc, re);
          tc::tmem_ld16(tim + cc, im);
          const int c0 = cbase + cc;
          if (LAY == LAY_SYM) {
            const int J = c0 >> 4;
            if (J >= I && r < 16 * mt) {
              S *tile = slot + (int64_t)(J * (J + 1) / 2 + I) * 256;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int c = c0 + i;
                const float2 v = (r < m && c < m) ? make_float2(re[i], im[i]) : make_float2(0.f, 0.f);
                if (J > I || i >= rr) tile[i * 16 + ((rr + i) & 15)] = store_c<S>(v);
                if (J == I && i > rr) tile[rr * 16 + ((i + rr) & 15)] = store_c<S>(v);
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = c0 + i;
              const float2 v = make_float2(re[i], im[i]);
              emit<S, LAY>(slot, r, c, v, m, ldm, mp8);
              if (top && c >= 128) emit<S, LAY>(slot, c, r, v, m, ldm, mp8);   // bottom-left block
            }
          }
          if (more) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = c0 + i;
              float2 v = make_float2(0.f, 0.f);
              if (r < m && c < m)
                v = cfms(cmul(lS[r], make_float2(re[i], im[i])), lS[c],
                         d_band<float2, float>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2));
              re[i] = v.x;
              im[i] = v.y;
            }
            tc::tmem_st16(tre + cc, re);
            tc::tmem_st16(tim + cc, im);
          }
        }
        tc::tmem_wait_st();
      }
    }
    __syncthreads();
    if (tid == 0) flags[box] = *sflag;
  }

  // ---- release tensor memory once no MMA is in flight
  tc::fence_before();
  __syncthreads();
  if (!alive && tid == 0) {
    tc::mma_commit(mbar);   // arrives when every MMA issued so far has completed
    volatile int never = 0;
    tc::bar_wait(mbar, nphase & 1u, &never);
  }
  __syncthreads();
  tc::fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FX_TMEM_COLS) : "memory");
}

template <typename S, int LAY>
static cudaError_t launch_tc(hd_ctx *ctx, void *factor, float tau2, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_factor_tc<S, LAY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(ctx->nsub, sms);   // one CTA per SM (tensor memory and shared memory both full)
  k_factor_tc<S, LAY><<<grid, FX_THREADS, kSmem, st>>>(ctx->d_subs, ctx->nsub, ctx->d_lpool, ctx->d_k2, ctx->NX,
                                                       ctx->h * ctx->h, reinterpret_cast<S *>(factor), tau2,
                                                       ctx->d_fflag, ctx->d_status);
  return cudaGetLastError();
}

bool factor_tc_supported(const hd_ctx *ctx) { return ctx->prec != HD_C128 && ctx->max_m <= FX_MAXM; }

cudaError_t launch_factor_tc(hd_ctx *ctx, void *factor, cudaStream_t st) {
  const float tau2 = (float)(ctx->fpivot * ctx->fpivot);
  if (ctx->tc) return launch_tc<float2, LAY_TC>(ctx, factor, tau2, st);
  if (ctx->prec == HD_C64)
    return ctx->sym ? launch_tc<float2, LAY_SYM>(ctx, factor, tau2, st) : launch_tc<float2, LAY_FULL>(ctx, factor, tau2, st);
  return ctx->sym ? launch_tc<__half2, LAY_SYM>(ctx, factor, tau2, st) : launch_tc<__half2, LAY_FULL>(ctx, factor, tau2, st);
}

}  // namespace hd
