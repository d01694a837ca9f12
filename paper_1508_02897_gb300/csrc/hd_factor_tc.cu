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

// (x0, x1) = h + m + l piecewise, BF16 pieces rounded to nearest (each remainder is
// exact in FP32), two values per conversion instruction; the pieces come packed as
// BF16 pairs (x0 in the low half).
__device__ __forceinline__ void split3x2(float x0, float x1, uint32_t &h, uint32_t &m, uint32_t &l) {
  const __nv_bfloat162 bh = __floats2bfloat162_rn(x0, x1);
  const float2 fh = __bfloat1622float2(bh);
  const float r0 = __fsub_rn(x0, fh.x), r1 = __fsub_rn(x1, fh.y);
  const __nv_bfloat162 bm = __floats2bfloat162_rn(r0, r1);
  const float2 fm = __bfloat1622float2(bm);
  const __nv_bfloat162 bl = __floats2bfloat162_rn(__fsub_rn(r0, fm.x), __fsub_rn(r1, fm.y));
  h = *reinterpret_cast<const uint32_t *>(&bh);
  m = *reinterpret_cast<const uint32_t *>(&bm);
  l = *reinterpret_cast<const uint32_t *>(&bl);
}

// Row r of an operand tile (16 BF16 values as 8 pairs) in the no-swizzle K-major layout:
// 8-row groups 256 bytes apart (SBO), the two 8-column core matrices 128 bytes apart (LBO).
__device__ __forceinline__ void put_row(unsigned char *tile, int r, const uint32_t *v) {
  unsigned char *p = tile + (r >> 3) * 256 + (r & 7) * 16;
  *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<uint4 *>(p + 128) = make_uint4(v[4], v[5], v[6], v[7]);
}

// Splits 16 values and writes the three pieces as row r of tiles t, t+1, t+2.
__device__ __forceinline__ void put_split(unsigned char *tiles, uint32_t tile_bytes, int t, int r, const float *v) {
  uint32_t h[8], m[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split3x2(v[2 * i], v[2 * i + 1], h[i], m[i], l[i]);
  put_row(tiles + (size_t)t * tile_bytes, r, h);
  put_row(tiles + (size_t)(t + 1) * tile_bytes, r, m);
  put_row(tiles + (size_t)(t + 2) * tile_bytes, r, l);
}

__device__ __forceinline__ float cabs2f(float2 a) { return a.x * a.x + a.y * a.y; }

// 1 / x for the pivots: the hardware approximation refined by one Newton step
// (r (2 - x r)), within about one ulp for normal x; a zero or non-finite x is caught by
// the pivot check before the result matters.
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * fmaf(-x, r, 2.f);
}

// Stored entry (r, c) of S_j^{-1} in the full or tensor-core layouts (zero outside m x m).
template <typename S, int LAY>
__device__ __forceinline__ void emit(S *slot, int r, int c, float2 v, int m, int ldm, int mp8) {
  if (LAY == LAY_FULL) {
    if (r < m && c < m) slot[(int64_t)c * ldm + r] = store_c<S>(v);
  } else {   // LAY_TC: chunk c/8, real then imaginary plane [mp8/8][2][8][4], TF32;
             // LAY_TC3: then the real and imaginary remainders, TF32
    if (r >= mp8 || c >= mp8) return;
    if (r >= m || c >= m) v = make_float2(0.f, 0.f);
    float *F = reinterpret_cast<float *>(slot);
    const int per = 8 * mp8;
    constexpr int NPL = LAY == LAY_TC3 ? 4 : 2;
    const int64_t o = (int64_t)(c >> 3) * NPL * per + (r >> 3) * 64 + ((c >> 2) & 1) * 32 + (r & 7) * 4 + (c & 3);
    const float hr = tf32_round(v.x), hi = tf32_round(v.y);
    F[o] = hr;
    F[o + per] = hi;
    if (LAY == LAY_TC3) {
      F[o + 2 * per] = tf32_round(v.x - hr);
      F[o + 3 * per] = tf32_round(v.y - hi);
    }
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
                                              : (LAY == LAY_TC    ? (int64_t)mp8 * mp8
                                                 : LAY == LAY_TC3 ? 2 * (int64_t)mp8 * mp8
                                                                  : (int64_t)m * s.ldm);
    const uint32_t idesc_top = tc::idesc_bf16(128, NP);
    const uint32_t idesc_bot = tc::idesc_bf16(128, NB > 0 ? NB : 16);

    // operand tiles and the panel copy start at zero: rows >= m are never written
    for (int i = tid; i < (int)(kOffG / 16); i += FX_THREADS)
      reinterpret_cast<uint4 *>(smem_raw)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) *sflag = 0;

    // ---- S_0 = D_0 into tensor memory (the three band entries of a row computed once)
    if (warp < 4 || (warp < 6 && mb > 0)) {
      const double *k2row = k2 + (int64_t)s.ey0 * NX + s.ex0;
      const bool top = warp < 4;
      const int r = tid;   // top: rows 0..127; warps 4, 5: rows 128 + (tid - 128)
      const int ncol = top ? NP : NB, cbase = top ? 0 : 128;
      const uint32_t tre = top ? tq : tq + 2 * NP, tim = top ? tq + NP : tq + 2 * NP + NB;
      float2 dband[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (r < m)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int c = r - 1 + t;
          if (c >= 0 && c < m) dband[t] = d_entry<float2, float>(r, c, 0, a1c, ia1f, a2c, ia2f, k2row, h2);
        }
      for (int cc = 0; cc < ncol; cc += 16) {
        float re[16], im[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int t = cbase + cc + i - r + 1;   // band position 0, 1, 2, or outside
          const float2 v = t == 0 ? dband[0] : (t == 1 ? dband[1] : (t == 2 ? dband[2] : make_float2(0.f, 0.f)));
          re[i] = v.x;
          im[i] = v.y;
        }
        tc::tmem_st16(tre + cc, re);
        tc::tmem_st16(tim + cc, im);
      }
    }
    tc::tmem_wait_st();

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

        // ---- B. the A operand, which needs C only: A = -X, X = C outside rows K and zero on
        //         rows K (their new values are stored directly), one row per thread; and the
        //         first pivot of the panel against every unprocessed row below the panel
        {
          const int r = tid, kr = r - k0;
          if (r < FX_ROWS && r < m) {
            const bool inK = kr >= 0 && kr < w;
            float vr[16], vi[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 c = Cs[r * CLD + i];
              vr[i] = inK ? 0.f : -c.x;
              vi[i] = inK ? 0.f : -c.y;
            }
            put_split(At, FX_ATILE, 0, r, vr);
            put_split(At, FX_ATILE, 3, r, vi);
            if (r >= k0 + w && !(cabs2f(Cs[k0 * CLD]) >= tau2 * cabs2f(Cs[r * CLD]))) *sflag = 1;
          }
        }
        // ---- P = C_K^{-1} (w x w) by Gauss-Jordan without pivoting, one entry per thread
        //      (i, jj) = (tid / 16, tid % 16), two alternating shared copies.  Two elimination
        //      steps k, k+1 per barrier: every thread loads the nine entries it needs and
        //      applies both in-place steps to its own entry (the same arithmetic as two
        //      separate steps).  Each pivot is checked by the threads of the unprocessed
        //      entries below it.
        {
          const int i = tid >> 4, jj = tid & 15;
          float2 *B0 = G, *B1 = G + 256;
          B0[tid] = (i < w && jj < w) ? Cs[(k0 + i) * CLD + jj] : make_float2(i == jj ? 1.f : 0.f, 0.f);
          __syncthreads();
          // in-place Gauss-Jordan value of entry (x, y) after the step with pivot index k and
          // inverse pivot ip: a_xy the entry, a_xk its pivot-column entry, a_ky its pivot-row entry
          auto gj = [](int x, int y, int k, float2 a_xy, float2 a_xk, float2 a_ky, float2 ip) -> float2 {
            if (x == k) return y == k ? ip : cmul(a_ky, ip);
            if (y == k) {
              const float2 v = cmul(a_xk, ip);
              return make_float2(-v.x, -v.y);
            }
            return cfms(a_xk, cmul(a_ky, ip), a_xy);
          };
          int par = 0;
#pragma unroll 1
          for (int k = 0; k < w; k += 2, par ^= 1) {
            const float2 *src = par ? B1 : B0;
            float2 *dst = par ? B0 : B1;
            const float2 piv = src[k * 16 + k], aik = src[i * 16 + k], akj = src[k * 16 + jj], aij = src[tid];
            const float p2 = cabs2f(piv);
            if (jj == k && i > k && i < w && !(p2 >= tau2 * cabs2f(aik))) *sflag = 1;
            if (tid == 0 && (!(p2 > 0.f) || !isfinite(p2))) *sflag = 1;
            const float rd = recip(p2);   // 1 / pivot = conj(pivot) / |pivot|^2
            const float2 ip = make_float2(piv.x * rd, -piv.y * rd);
            float2 v = gj(i, jj, k, aij, aik, akj, ip);
            const int k1 = k + 1;
            if (k1 < w) {
              // the second step on the values after the first
              const float2 a_i1 = src[i * 16 + k1], a_k1 = src[k * 16 + k1];
              const float2 a_1j = src[k1 * 16 + jj], a_1k = src[k1 * 16 + k], a_11 = src[k1 * 16 + k1];
              const float2 vi1 = gj(i, k1, k, a_i1, aik, a_k1, ip);     // entry (i, k+1)
              const float2 v1j = gj(k1, jj, k, a_1j, a_1k, akj, ip);    // entry (k+1, jj)
              const float2 piv1 = gj(k1, k1, k, a_11, a_1k, a_k1, ip);  // next pivot
              const float q2 = cabs2f(piv1);
              if (jj == k1 && i > k1 && i < w && !(q2 >= tau2 * cabs2f(vi1))) *sflag = 1;
              if (tid == 0 && (!(q2 > 0.f) || !isfinite(q2))) *sflag = 1;
              const float rd1 = recip(q2);
              const float2 ip1 = make_float2(piv1.x * rd1, -piv1.y * rd1);
              v = gj(i, jj, k1, v, vi1, v1j, ip1);
            }
            dst[tid] = v;
            __syncthreads();
          }
          // P into the first copy, zero outside w x w
          const float2 *res = par ? B1 : B0;
          const float2 pv = (i < w && jj < w) ? res[tid] : make_float2(0.f, 0.f);
          __syncthreads();
          B0[tid] = pv;
          __syncthreads();
        }
        const float2 *Pm = G;   // P[i][kk] at Pm[i * 16 + kk], zero outside w x w

        // ---- C. the B operand Y^T = Z P (three BF16 pieces); Y^T also replaces C in the panel copy
        if (tid < FX_ROWS && tid < m) {
          const int r = tid, kr = r - k0;
          const bool inK = kr >= 0 && kr < w;
          float vr[16], vi[16];
          float2 y[16];
          if (inK) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) y[kk] = Pm[kr * 16 + kk];
          } else {
            // y = zs C[r] P: q outer, 16 independent accumulator chains
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) y[kk] = make_float2(0.f, 0.f);
            // kept as a loop over q (16 independent accumulators per step): a fully
            // unrolled copy is 1024 FMAs of straight-line code in an already large kernel
#pragma unroll 1
            for (int q = 0; q < 16; ++q) {
              const float4 *prow = reinterpret_cast<const float4 *>(Pm + q * 16);
              const float2 cq = Cs[r * CLD + q];
#pragma unroll
              for (int k2 = 0; k2 < 8; ++k2) {
                const float4 pp = prow[k2];
                y[2 * k2] = cfma(cq, make_float2(pp.x, pp.y), y[2 * k2]);
                y[2 * k2 + 1] = cfma(cq, make_float2(pp.z, pp.w), y[2 * k2 + 1]);
              }
            }
            if (r < k0)
#pragma unroll
              for (int kk = 0; kk < 16; ++kk) y[kk] = make_float2(-y[kk].x, -y[kk].y);
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
          const int q = warp & 3;
          const bool top_rmw = k0 < 128 && q == (k0 >> 5);
          const bool bot_rmw = k0 >= 128 && q == ((k0 - 128) >> 5);
          // columns K of rows outside K: zero (top rows: warps 0-3; bottom rows: warps 4, 5)
          if (warp < 4 && !top_rmw) {
            const float z[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            tc::tmem_st16(tq + k0, z);
            tc::tmem_st16(tq + NP + k0, z);
          } else if ((warp == 4 || warp == 5) && k0 >= 128 && !bot_rmw) {
            const float z[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            tc::tmem_st16(tq + 2 * NP + (k0 - 128), z);
            tc::tmem_st16(tq + 2 * NP + NB + (k0 - 128), z);
          }
          if (top_rmw || bot_rmw) {
            // the two warps of this lane quarter rewrite the rows of K, half the columns each
            const int rrow = top_rmw ? 32 * q + lane : 128 + 32 * q + lane;
            const int kr = rrow - k0;
            const bool inK = kr >= 0 && kr < w;
            const int ncol = top_rmw ? NP : NB, cb = top_rmw ? 0 : 128, kc = k0 - cb;
            const int nch = ncol / 16, half = (nch + 1) / 2;
            const int ch0 = warp < 4 ? 0 : half, ch1 = warp < 4 ? half : nch;
            const uint32_t tre = top_rmw ? tq : tq + 2 * NP, tim = top_rmw ? tq + NP : tq + 2 * NP + NB;
            for (int c2 = ch0; c2 < ch1; c2 += 2) {
              float re[2][16], im[2][16];
              const int nh = c2 + 1 < ch1 ? 2 : 1;   // chunks of 16 columns in this pass, one wait
              for (int hh = 0; hh < nh; ++hh) {
                tc::tmem_ld16_nw(tre + 16 * (c2 + hh), re[hh]);
                tc::tmem_ld16_nw(tim + 16 * (c2 + hh), im[hh]);
              }
              tc::tmem_wait_ld();
              for (int hh = 0; hh < nh; ++hh) {
                const int cc = 16 * (c2 + hh);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  if (inK) {
                    const float2 v = Cs[(cb + cc + i) * CLD + kr];
                    re[hh][i] = v.x;
                    im[hh][i] = v.y;
                  } else if (cc == kc) {
                    re[hh][i] = 0.f;
                    im[hh][i] = 0.f;
                  }
                }
                tc::tmem_st16(tre + cc, re[hh]);
                tc::tmem_st16(tim + cc, im[hh]);
              }
            }
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
        const bool ok = tc::bar_spin(mbar, nphase & 1u, abort_flag);
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
      // every warp takes part: warps 0-3 the left columns of their rows 0..127, warps 4-7 the
      // right columns of the same rows, warps 4 and 5 also the bottom-right block (rows
      // 128..m-1), the column split balancing the 16-column chunks
      {
        const int q = warp & 3;
        const int nchT = NP / 16, nchB = NB / 16, sT = (nchT + nchB + 1) / 2;
        for (int reg = 0; reg < 2; ++reg) {
          const bool top = reg == 0;
          int ch0, ch1;
          if (top) {
            ch0 = warp < 4 ? 0 : min(sT, nchT);
            ch1 = warp < 4 ? min(sT, nchT) : nchT;
          } else {
            ch0 = 0;
            ch1 = (warp == 4 || warp == 5) ? nchB : 0;
          }
          if (ch0 >= ch1) continue;
          const int r = top ? 32 * q + lane : 128 + 32 * q + lane;
          const int cbase = top ? 0 : 128;
          const uint32_t tre = top ? tq : tq + 2 * NP, tim = top ? tq + NP : tq + 2 * NP + NB;
          const int I = r >> 4, rr = r & 15;
          // the three entries of D_{j+1} in row r (west, centre, east), once per row
          float2 dband[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          const float2 lr = lS[r];
          if (more && r < m)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const int c = r - 1 + t;
              if (c >= cbase + 16 * ch0 - 1 && c <= cbase + 16 * ch1 && c >= 0 && c < m)
                dband[t] = d_entry<float2, float>(r, c, j + 1, a1c, ia1f, a2c, ia2f, k2row, h2);
            }
          for (int c2 = ch0; c2 < ch1; c2 += 2) {
            float rb[2][16], ib[2][16];
            const int nh = c2 + 1 < ch1 ? 2 : 1;   // chunks of 16 columns in this pass, one wait
            for (int hh = 0; hh < nh; ++hh) {
              tc::tmem_ld16_nw(tre + 16 * (c2 + hh), rb[hh]);
              tc::tmem_ld16_nw(tim + 16 * (c2 + hh), ib[hh]);
            }
            tc::tmem_wait_ld();
            for (int hh = 0; hh < nh; ++hh) {
              const int cc = 16 * (c2 + hh);
              float *re = rb[hh], *im = ib[hh];
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
                  if (r < m && c < m) {
                    const int t = c - r + 1;   // band position 0, 1, 2, or outside
                    const float2 d = t == 0 ? dband[0] : (t == 1 ? dband[1] : (t == 2 ? dband[2] : make_float2(0.f, 0.f)));
                    v = cfms(cmul(lr, make_float2(re[i], im[i])), lS[c], d);
                  }
                  re[i] = v.x;
                  im[i] = v.y;
                }
                tc::tmem_st16(tre + cc, re);
                tc::tmem_st16(tim + cc, im);
              }
            }
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
  cudaError_t e = allow_smem(k_factor_tc<S, LAY>, kSmem);
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
  if (ctx->tc3) return launch_tc<float2, LAY_TC3>(ctx, factor, tau2, st);
  if (ctx->tc) return launch_tc<float2, LAY_TC>(ctx, factor, tau2, st);
  if (ctx->prec == HD_C64)
    return ctx->sym ? launch_tc<float2, LAY_SYM>(ctx, factor, tau2, st) : launch_tc<float2, LAY_FULL>(ctx, factor, tau2, st);
  if (ctx->prec == HD_C64_B)
    return ctx->sym ? launch_tc<__nv_bfloat162, LAY_SYM>(ctx, factor, tau2, st)
                    : launch_tc<__nv_bfloat162, LAY_FULL>(ctx, factor, tau2, st);
  return ctx->sym ? launch_tc<__half2, LAY_SYM>(ctx, factor, tau2, st) : launch_tc<__half2, LAY_FULL>(ctx, factor, tau2, st);
}

}  // namespace hd
