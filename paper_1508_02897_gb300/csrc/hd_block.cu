// Block flexible GMRES: p right-hand sides sharing one Krylov space (the outer solver
// of Sec. 3 taken to many sources at once; the block method is the textbook one, Saad,
// "Iterative Methods for Sparse Linear Systems", 2nd ed., Sec. 6.12, made flexible as in
// Sec. 9.4, with block classical Gram-Schmidt twice as in the point FGMRES).
//
// Per cycle: R = B - A X and R = V_0 S (thin QR); block step j: Z_j = M V_j (the
// one-step preconditioner applied to the p columns in one launch), W = A Z_j,
// H_ij = V_i^H W for all i <= j from the same W and W -= sum_i V_i H_ij, the pass done
// twice, then W = V_{j+1} H_{j+1,j} (thin QR).  The least squares on the block
// Hessenberg matrix (min || E_1 S - Hbar Y ||_F) is kept as an incremental Householder
// QR on the host, which gives every column's residual estimate after each step; the
// cycle ends when every column's estimate is <= rtol, at the restart, or when a new
// block loses a direction to rounding; then X += [Z_0 .. Z_k] Y and the FP64 true
// residual decides whether to start another cycle.
//
// Device arithmetic: the preconditioner in the context's precision, everything else in
// FP64.  The dense block operations are two kernels: a Gram kernel (sums of
// conj(A_i) B_c over all elements, per-block partial sums reduced in a fixed order, so
// results are reproducible) and a combination kernel (OUT_c = IN_c + sum_i A_i M_ic).
// The thin QR is Cholesky QR done twice (CholQR2): G = W^H W on the device, its
// Cholesky factor and inverse on the host, W R^-1 on the device, repeated once more;
// R = R2 R1 is upper triangular with a real positive diagonal.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "hd_internal.cuh"

namespace hd {

namespace {

using cd = std::complex<double>;

constexpr int BG_T = 256;   // threads per block of the block kernels
constexpr int BG_TI = 4;    // A vectors per Gram tile
constexpr int BG_TC = 4;    // B vectors per Gram tile
constexpr int BC_TC = 8;    // output columns per combination tile
constexpr int BC_KI = 32;   // A vectors staged per shared-memory pass of the combination

__device__ __forceinline__ double2 dconj_mul(double2 a, double2 b) {   // conj(a) b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// partial[blk][i][c] = sum over this block's elements e of conj(A_i[e]) B_c[e], for the
// tile i in [ti, ti + BG_TI), c in [tc, tc + BG_TC) (grid.y, grid.z); elements are taken
// grid-stride by the grid.x blocks.
__global__ void __launch_bounds__(BG_T) k_bgram(const double2 *__restrict__ A, int64_t lda, int na,
                                                const double2 *__restrict__ Bv, int64_t ldb, int nb, int64_t n,
                                                double2 *__restrict__ partial) {
  const int ti = blockIdx.y * BG_TI, tc = blockIdx.z * BG_TC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2 acc[BG_TI][BG_TC];
#pragma unroll
  for (int a = 0; a < BG_TI; ++a)
#pragma unroll
    for (int b = 0; b < BG_TC; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int64_t e = (int64_t)blockIdx.x * BG_T + tid; e < n; e += (int64_t)gridDim.x * BG_T) {
    double2 av[BG_TI], bv[BG_TC];
#pragma unroll
    for (int a = 0; a < BG_TI; ++a) av[a] = ti + a < na ? A[(int64_t)(ti + a) * lda + e] : make_double2(0.0, 0.0);
#pragma unroll
    for (int b = 0; b < BG_TC; ++b) bv[b] = tc + b < nb ? Bv[(int64_t)(tc + b) * ldb + e] : make_double2(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < BG_TI; ++a)
#pragma unroll
      for (int b = 0; b < BG_TC; ++b) {
        const double2 p = dconj_mul(av[a], bv[b]);
        acc[a][b].x += p.x;
        acc[a][b].y += p.y;
      }
  }
  __shared__ double2 red[BG_T / 32][BG_TI * BG_TC];
#pragma unroll
  for (int a = 0; a < BG_TI; ++a)
#pragma unroll
    for (int b = 0; b < BG_TC; ++b) {
      double x = acc[a][b].x, y = acc[a][b].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == 0) red[warp][a * BG_TC + b] = make_double2(x, y);
    }
  __syncthreads();
  if (tid < BG_TI * BG_TC) {
    const int a = tid / BG_TC, b = tid % BG_TC;
    double2 s = red[0][tid];
    for (int w = 1; w < BG_T / 32; ++w) {
      s.x += red[w][tid].x;
      s.y += red[w][tid].y;
    }
    if (ti + a < na && tc + b < nb) partial[((int64_t)blockIdx.x * na + ti + a) * nb + tc + b] = s;
  }
}

// out[k] = sum over the G blocks of partial[blk][k] (k < count), in block order.
__global__ void k_breduce(const double2 *__restrict__ partial, int G, int count, double2 *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  double2 s = make_double2(0.0, 0.0);
  for (int g = 0; g < G; ++g) {
    const double2 v = partial[(int64_t)g * count + k];
    s.x += v.x;
    s.y += v.y;
  }
  out[k] = s;
}

// OUT_c[e] = (IN ? IN_c[e] : 0) + sum_{i < na} A_i[e] M[i][c] for the columns
// c in [tc, tc + BC_TC) (grid.y); M is na x nb complex, row-major.  OUT may be IN (each
// element is read before it is written by the same thread) but not one of the A_i.
__global__ void __launch_bounds__(BG_T) k_bcomb(const double2 *__restrict__ A, int64_t lda, int na,
                                                const double2 *__restrict__ M, int nb, const double2 *IN,
                                                int64_t ldin, double2 *OUT, int64_t ldout, int64_t n) {
  __shared__ double2 ms[BC_KI][BC_TC];
  const int tc = blockIdx.y * BC_TC;
  const int ncol = min(BC_TC, nb - tc);
  for (int64_t e0 = (int64_t)blockIdx.x * BG_T; e0 < n; e0 += (int64_t)gridDim.x * BG_T) {
    const int64_t e = e0 + threadIdx.x;
    double2 acc[BC_TC];
#pragma unroll
    for (int c = 0; c < BC_TC; ++c)
      acc[c] = (IN && c < ncol && e < n) ? IN[(int64_t)(tc + c) * ldin + e] : make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < na; i0 += BC_KI) {
      const int ki = min(BC_KI, na - i0);
      __syncthreads();
      for (int q = threadIdx.x; q < BC_KI * BC_TC; q += BG_T) {
        const int i = q / BC_TC, c = q % BC_TC;
        ms[i][c] = (i < ki && c < ncol) ? M[(int64_t)(i0 + i) * nb + tc + c] : make_double2(0.0, 0.0);
      }
      __syncthreads();
      if (e < n)
        for (int i = 0; i < ki; ++i) {
          const double2 a = A[(int64_t)(i0 + i) * lda + e];
#pragma unroll
          for (int c = 0; c < BC_TC; ++c) {
            const double2 m = ms[i][c];
            acc[c].x = fma(a.x, m.x, fma(-a.y, m.y, acc[c].x));
            acc[c].y = fma(a.x, m.y, fma(a.y, m.x, acc[c].y));
          }
        }
    }
    if (e < n)
#pragma unroll
      for (int c = 0; c < BC_TC; ++c)
        if (c < ncol) OUT[(int64_t)(tc + c) * ldout + e] = acc[c];
  }
}

// ---------------------------------------------------------------- host linear algebra (FP64)
// Upper-triangular R with G = R^H R for a Hermitian p x p matrix G (row-major); false when
// a pivot is not positive (the block has lost a direction).
bool cholesky_upper(const std::vector<cd> &G, int p, std::vector<cd> &R) {
  R.assign((size_t)p * p, cd(0.0, 0.0));
  for (int i = 0; i < p; ++i) {
    double d = G[(size_t)i * p + i].real();
    for (int k = 0; k < i; ++k) d -= std::norm(R[(size_t)k * p + i]);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double rii = std::sqrt(d);
    R[(size_t)i * p + i] = rii;
    for (int j = i + 1; j < p; ++j) {
      cd sum = G[(size_t)i * p + j];
      for (int k = 0; k < i; ++k) sum -= std::conj(R[(size_t)k * p + i]) * R[(size_t)k * p + j];
      R[(size_t)i * p + j] = sum / rii;
    }
  }
  return true;
}

// Inverse of an upper-triangular p x p matrix (row-major).
std::vector<cd> inv_upper(const std::vector<cd> &R, int p) {
  std::vector<cd> X((size_t)p * p, cd(0.0, 0.0));
  for (int c = 0; c < p; ++c) {
    X[(size_t)c * p + c] = 1.0 / R[(size_t)c * p + c];
    for (int i = c - 1; i >= 0; --i) {
      cd sum(0.0, 0.0);
      for (int k = i + 1; k <= c; ++k) sum += R[(size_t)i * p + k] * X[(size_t)k * p + c];
      X[(size_t)i * p + c] = -sum / R[(size_t)i * p + i];
    }
  }
  return X;
}

// A (m x k) B (k x n), row-major.
std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, int m, int k, int n) {
  std::vector<cd> C((size_t)m * n, cd(0.0, 0.0));
  for (int i = 0; i < m; ++i)
    for (int q = 0; q < k; ++q) {
      const cd a = A[(size_t)i * k + q];
      for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)q * n + j];
    }
  return C;
}

// min || E_1 S - Hbar Y ||_F over a block upper Hessenberg Hbar ((k+1)p x kp, the blocks
// under the diagonal upper triangular), kept as an incremental Householder QR: column c
// has nonzeros down to row c + p, so its reflector spans rows c .. c + p.  After block
// column j is added, the rows (j+1)p .. (j+2)p - 1 of the transformed right-hand side
// are the residual of each column.
struct BlockLS {
  int p = 0, R = 0, ld = 0, k = 0;
  std::vector<cd> H;     // ld x (R p), column-major (triangularised)
  std::vector<cd> g;     // ld x p, column-major (transformed right-hand side)
  std::vector<cd> v;     // (R p) reflectors of p + 1 entries
  std::vector<cd> tau;

  void init(int p_, int R_, const std::vector<cd> &S) {   // S: p x p row-major
    p = p_;
    R = R_;
    ld = (R + 1) * p;
    k = 0;
    H.assign((size_t)ld * R * p, cd(0.0, 0.0));
    g.assign((size_t)ld * p, cd(0.0, 0.0));
    v.assign((size_t)R * p * (p + 1), cd(0.0, 0.0));
    tau.assign((size_t)R * p, cd(0.0, 0.0));
    for (int i = 0; i < p; ++i)
      for (int c = 0; c < p; ++c) g[(size_t)c * ld + i] = S[(size_t)i * p + c];
  }
  // y[rows c .. c+p] -= tau v (v^H y)
  void reflect(int c, cd *y) const {
    const cd *vc = &v[(size_t)c * (p + 1)];
    cd s(0.0, 0.0);
    for (int q = 0; q <= p; ++q) s += std::conj(vc[q]) * y[c + q];
    s *= tau[c];
    for (int q = 0; q <= p; ++q) y[c + q] -= s * vc[q];
  }
  // Block column j = k: hc is ((j+2)p) x p row-major (the coefficients H_ij and H_{j+1,j}).
  void add(const std::vector<cd> &hc) {
    const int j = k, rows = (j + 2) * p;
    for (int t = 0; t < p; ++t) {
      cd *col = &H[(size_t)(j * p + t) * ld];
      for (int i = 0; i < ld; ++i) col[i] = i < rows ? hc[(size_t)i * p + t] : cd(0.0, 0.0);
      for (int c = 0; c < j * p + t; ++c) reflect(c, col);   // earlier reflectors, in order
      // new reflector for column c = jp + t on rows c .. c + p
      const int c = j * p + t;
      cd *vc = &v[(size_t)c * (p + 1)];
      double nx = 0.0;
      for (int q = 0; q <= p; ++q) nx += std::norm(col[c + q]);
      nx = std::sqrt(nx);
      const cd x0 = col[c];
      if (nx == 0.0) {
        tau[c] = 0.0;
        for (int q = 0; q <= p; ++q) vc[q] = 0.0;
        continue;
      }
      const cd alpha = (std::abs(x0) > 0.0 ? -x0 / std::abs(x0) : cd(-1.0, 0.0)) * nx;
      for (int q = 0; q <= p; ++q) vc[q] = col[c + q];
      vc[0] -= alpha;
      double vn = 0.0;
      for (int q = 0; q <= p; ++q) vn += std::norm(vc[q]);
      tau[c] = vn > 0.0 ? 2.0 / vn : 0.0;
      col[c] = alpha;
      for (int q = 1; q <= p; ++q) col[c + q] = 0.0;
      for (int c2 = 0; c2 < p; ++c2) reflect(c, &g[(size_t)c2 * ld]);
    }
    ++k;
  }
  double residual(int c) const {   // of right-hand side c after the last added block
    double s = 0.0;
    for (int i = k * p; i < (k + 1) * p; ++i) s += std::norm(g[(size_t)c * ld + i]);
    return std::sqrt(s);
  }
  // Y (k p x p, row-major) from the triangle of the first k block columns
  std::vector<cd> solve() const {
    const int m = k * p;
    std::vector<cd> Y((size_t)m * p, cd(0.0, 0.0));
    for (int c = 0; c < p; ++c)
      for (int i = m - 1; i >= 0; --i) {
        cd s = g[(size_t)c * ld + i];
        for (int q = i + 1; q < m; ++q) s -= H[(size_t)q * ld + i] * Y[(size_t)q * p + c];
        Y[(size_t)i * p + c] = s / H[(size_t)i * ld + i];
      }
    return Y;
  }
};

// ---------------------------------------------------------------- device helpers
struct BlockWs {
  int64_t n;
  int p, R, GB;
  double2 *V, *Z, *T, *partial, *out, *coef;
};

int block_gram_blocks() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 4 * sms;
}

BlockWs block_layout(void *kws, int64_t n, int p, int R, int GB) {
  BlockWs w;
  w.n = n; w.p = p; w.R = R; w.GB = GB;
  double2 *b = reinterpret_cast<double2 *>(kws);
  w.V = b; b += (int64_t)(R + 1) * p * n;
  w.Z = b; b += (int64_t)R * p * n;
  w.T = b; b += (int64_t)p * n;
  w.partial = b; b += (int64_t)GB * (R + 1) * p * p;
  w.out = b; b += (int64_t)(R + 1) * p * p;
  w.coef = b;
  return w;
}

size_t block_bytes(int64_t n, int p, int R, int GB) {
  return sizeof(double2) * ((size_t)(2 * R + 2) * p * n + (size_t)GB * (R + 1) * p * p + 2 * (size_t)(R + 1) * p * p);
}

// host G (na x nb, row-major) = A^H B over the n elements (A: na vectors, B: nb vectors)
int gram(hd_ctx *ctx, const BlockWs &w, const double2 *A, int na, const double2 *Bv, int nb, std::vector<cd> &G,
         cudaStream_t st) {
  dim3 grid(w.GB, (na + BG_TI - 1) / BG_TI, (nb + BG_TC - 1) / BG_TC);
  k_bgram<<<grid, BG_T, 0, st>>>(A, w.n, na, Bv, w.n, nb, w.n, w.partial);
  const int cnt = na * nb;
  k_breduce<<<(cnt + 255) / 256, 256, 0, st>>>(w.partial, w.GB, cnt, w.out);
  ctx->t_launch[T_ARNOLDI] += 2;
  G.resize((size_t)cnt);
  cudaError_t e = cudaMemcpyAsync(G.data(), w.out, sizeof(double2) * cnt, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "block Gram");
  return HD_OK;
}

// OUT = (IN or 0) + A M, M host (na x nb, row-major)
int combine(hd_ctx *ctx, const BlockWs &w, const double2 *A, int na, const std::vector<cd> &M, int nb,
            const double2 *IN, double2 *OUT, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(w.coef, M.data(), sizeof(double2) * (size_t)na * nb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "block coefficients");
  const int gx = (int)std::min<int64_t>((w.n + BG_T - 1) / BG_T, 1 << 20);
  dim3 grid(gx, (nb + BC_TC - 1) / BC_TC);
  k_bcomb<<<grid, BG_T, 0, st>>>(A, w.n, na, w.coef, nb, IN, w.n, OUT, w.n, w.n);
  ctx->t_launch[T_ARNOLDI] += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "block combination");
  return HD_OK;
}

// Thin QR of the p columns of IN by CholQR2: OUT = IN R^-1 with R (p x p, upper) returned;
// TMP holds the intermediate basis.  false (and R from the first Cholesky, its failed
// pivots zero) when the block has lost a direction.
int cholqr2(hd_ctx *ctx, const BlockWs &w, const double2 *IN, double2 *TMP, double2 *OUT, std::vector<cd> &R,
            bool &ok, cudaStream_t st) {
  const int p = w.p;
  std::vector<cd> G, R1, R2;
  int rc = gram(ctx, w, IN, p, IN, p, G, st);
  if (rc) return rc;
  ok = cholesky_upper(G, p, R1);
  if (!ok) {
    R = R1;   // the pivots up to the failure; the rest zero
    return HD_OK;
  }
  rc = combine(ctx, w, IN, p, inv_upper(R1, p), p, nullptr, TMP, st);
  if (!rc) rc = gram(ctx, w, TMP, p, TMP, p, G, st);
  if (rc) return rc;
  ok = cholesky_upper(G, p, R2);
  if (!ok) {
    R = R1;
    return HD_OK;
  }
  rc = combine(ctx, w, TMP, p, inv_upper(R2, p), p, nullptr, OUT, st);
  R = matmul(R2, R1, p, p, p);
  return rc;
}

}  // namespace

size_t block_krylov_bytes(int64_t n, int restart, int p) { return block_bytes(n, p, restart, block_gram_blocks()); }

int run_block_gmres(hd_ctx *ctx, const double2 *b, double2 *x, int p, const hd_gmres_opts *o, void *kws,
                    void *scratch, hd_gmres_stats *stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const int R = o->restart;
  const int64_t n = (int64_t)ctx->NX * ctx->NY;
  const BlockWs w = block_layout(kws, n, p, R, block_gram_blocks());
  double2 *V = w.V, *Z = w.Z, *T = w.T;
  auto Vb = [&](int j) { return V + (int64_t)j * p * n; };
  auto Zb = [&](int j) { return Z + (int64_t)j * p * n; };
  std::vector<cd> G;
  int rc = gram(ctx, w, b, p, b, p, G, st);   // ||b_c||^2 on the diagonal
  if (rc) return rc;
  std::vector<double> bnorm(p), truer(p, 1.0), est(p, 1.0);
  for (int c = 0; c < p; ++c) bnorm[c] = std::sqrt(std::max(G[(size_t)c * p + c].real(), 0.0));
  if (!o->use_x0) {
    cudaError_t e = cudaMemsetAsync(x, 0, sizeof(double2) * (size_t)p * n, st);
    if (e != cudaSuccess) return cuda_fail(e, "block GMRES start");
  }
  int iters = 0, cycles = 0;
  bool numeric = false;
  BlockLS ls;
  while (true) {
    // R = B - A X (B itself for the first cycle from zero) into T
    cudaError_t e = (cycles > 0 || o->use_x0) ? launch_residual_strided(ctx, b, n, x, n, T, n, p, st)
                                              : cudaMemcpyAsync(T, b, sizeof(double2) * (size_t)p * n,
                                                                cudaMemcpyDeviceToDevice, st);
    ctx->t_launch[T_MATVEC] += (cycles > 0 || o->use_x0) ? 1 : 0;
    if (e != cudaSuccess) return cuda_fail(e, "block GMRES residual");
    rc = gram(ctx, w, T, p, T, p, G, st);
    if (rc) return rc;
    bool all = true;
    for (int c = 0; c < p; ++c) {
      truer[c] = bnorm[c] > 0.0 ? std::sqrt(std::max(G[(size_t)c * p + c].real(), 0.0)) / bnorm[c] : 0.0;
      all = all && truer[c] <= o->rtol;
    }
    if (all || iters >= o->max_iters || numeric) break;
    // R = V_0 S: T -> V_1 (intermediate) -> V_0
    std::vector<cd> S;
    bool ok = true;
    rc = cholqr2(ctx, w, T, Vb(R >= 1 ? 1 : 0), Vb(0), S, ok, st);
    if (rc) return rc;
    if (!ok) {   // the residual block itself is rank deficient (for example two equal sources)
      set_error("hd_block_gmres_solve: the residual block is rank deficient; solve dependent sources separately");
      return HD_ERR_NUMERIC;
    }
    ls.init(p, R, S);
    int k = 0;
    for (int j = 0; j < R; ++j) {
      // Z_j = M V_j (the p columns in one preconditioner launch), W = A Z_j into V_{j+1}
      rc = run_apply(ctx, Vb(j), n, Zb(j), n, p, scratch, st);
      if (rc) return rc;
      tic(ctx, T_MATVEC, st);
      e = launch_matvec(ctx, Zb(j), n, Vb(j + 1), n, p, st);
      toc(ctx, T_MATVEC, st, 1);
      if (e != cudaSuccess) return cuda_fail(e, "block GMRES matvec");
      // block classical Gram-Schmidt, twice; the first Gram also gives ||W||_F
      tic(ctx, T_ARNOLDI, st);
      std::vector<cd> Hc((size_t)(j + 2) * p * p, cd(0.0, 0.0));
      const int na = (j + 1) * p;
      double wnorm2 = 0.0;
      for (int pass = 0; pass < 2 && !rc; ++pass) {
        rc = gram(ctx, w, V, pass == 0 ? na + p : na, Vb(j + 1), p, G, st);
        if (rc) break;
        if (pass == 0)
          for (int c = 0; c < p; ++c) wnorm2 += G[(size_t)(na + c) * p + c].real();
        std::vector<cd> M((size_t)na * p);
        for (int i = 0; i < na; ++i)
          for (int c = 0; c < p; ++c) {
            Hc[(size_t)i * p + c] += G[(size_t)i * p + c];
            M[(size_t)i * p + c] = -G[(size_t)i * p + c];
          }
        rc = combine(ctx, w, V, na, M, p, Vb(j + 1), Vb(j + 1), st);
      }
      // W = V_{j+1} H_{j+1,j}: V_{j+1} -> T -> V_{j+1}
      std::vector<cd> Hn;
      if (!rc) rc = cholqr2(ctx, w, Vb(j + 1), T, Vb(j + 1), Hn, ok, st);
      toc(ctx, T_ARNOLDI, st, 0);
      if (rc) return rc;
      for (int i = 0; i < p; ++i)
        for (int c = 0; c < p; ++c) Hc[(size_t)(na + i) * p + c] = Hn[(size_t)i * p + c];
      ls.add(Hc);
      ++iters;
      k = j + 1;
      bool conv = true;
      for (int c = 0; c < p; ++c) {
        est[c] = bnorm[c] > 0.0 ? ls.residual(c) / bnorm[c] : 0.0;
        conv = conv && est[c] <= o->rtol;
        if (!std::isfinite(est[c])) numeric = true;
      }
      // a direction of the new block cancelled to rounding: the block space stops growing
      double dmin = 1e300;
      for (int i = 0; i < p; ++i) dmin = std::min(dmin, std::abs(Hn[(size_t)i * p + i]));
      const bool deficient = !ok || dmin <= 1e-12 * std::max(std::sqrt(wnorm2), 1e-300);
      if (conv || deficient || numeric || iters >= o->max_iters) break;
    }
    // X += [Z_0 .. Z_{k-1}] Y
    std::vector<cd> Y = ls.solve();
    for (const cd &yv : Y)
      if (!std::isfinite(yv.real()) || !std::isfinite(yv.imag())) numeric = true;
    if (numeric) break;
    tic(ctx, T_ARNOLDI, st);
    rc = combine(ctx, w, Z, k * p, Y, p, x, x, st);
    toc(ctx, T_ARNOLDI, st, 0);
    if (rc) return rc;
    ++cycles;
  }
  const double ts = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool allc = true;
  for (int c = 0; c < p; ++c) {
    hd_gmres_stats &sc = stats[c];
    sc.iters = iters;
    sc.restarts = cycles;
    sc.converged = truer[c] <= o->rtol ? 1 : 0;
    sc.status = numeric ? HD_ERR_NUMERIC : (sc.converged ? HD_OK : HD_ERR_NOT_CONVERGED);
    sc.relres_est = est[c];
    sc.relres_true = truer[c];
    sc.t_solve_s = ts;
    sc.second_passes = iters;
    sc.second_pass_vecs = 0;
    allc = allc && sc.converged;
  }
  if (numeric) {
    set_error("hd_block_gmres_solve: non-finite value in the block Arnoldi process");
    return HD_ERR_NUMERIC;
  }
  return allc ? HD_OK : HD_ERR_NOT_CONVERGED;
}

}  // namespace hd

using namespace hd;

extern "C" {

int hd_query_block_workspace(const hd_ctx *c, int32_t p, int32_t restart, size_t *krylov_bytes,
                             size_t *scratch_bytes) {
  if (!c || p < 1 || p > HD_MAX_BLOCK || restart < 1 || restart > HD_MAX_RESTART) {
    set_error("hd_query_block_workspace: bad context, block size (1 .. HD_MAX_BLOCK) or restart");
    return HD_ERR_INVALID;
  }
  if (krylov_bytes) *krylov_bytes = block_krylov_bytes((int64_t)c->NX * c->NY, restart, p);
  if (scratch_bytes)
    *scratch_bytes = compute_bytes(c->prec) * (size_t)std::max(c->staging_elems * (int64_t)p, c->work_elems);
  return HD_OK;
}

int hd_block_gmres_solve(hd_ctx *c, const void *b, void *x, int32_t p, const hd_gmres_opts *o, void *kws,
                         size_t kbytes, void *scratch, size_t scratch_bytes, hd_gmres_stats *stats, void *stream) {
  if (!o || o->restart < 1 || o->restart > HD_MAX_RESTART || o->max_iters < 0 || !(o->rtol >= 0) ||
      o->precond_steps > 1 || o->precond_steps < 0) {
    set_error("hd_block_gmres_solve: bad options (the one-step preconditioner only)");
    return HD_ERR_INVALID;
  }
  if (!c || !b || !x || !kws || !scratch || !stats || p < 1 || p > HD_MAX_BLOCK) {
    set_error("hd_block_gmres_solve: bad argument");
    return HD_ERR_INVALID;
  }
  if (!c->factored) {
    set_error("hd_block_gmres_solve: call hd_factor_subdomains first");
    return HD_ERR_INVALID;
  }
  size_t kb = 0, sb = 0;
  hd_query_block_workspace(c, p, o->restart, &kb, &sb);
  if (kbytes < kb || scratch_bytes < sb) {
    set_error("hd_block_gmres_solve: workspace too small (hd_query_block_workspace)");
    return HD_ERR_OOM;
  }
  auto a16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  if (!a16(b) || !a16(x) || !a16(kws) || !a16(scratch)) {
    set_error("hd_block_gmres_solve: buffers must be 16-byte aligned");
    return HD_ERR_INVALID;
  }
  std::memset(stats, 0, sizeof(hd_gmres_stats) * p);
  return run_block_gmres(c, reinterpret_cast<const double2 *>(b), reinterpret_cast<double2 *>(x), p, o, kws, scratch,
                         stats, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
