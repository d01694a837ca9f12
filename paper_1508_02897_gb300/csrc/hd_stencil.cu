// Medium and PML tables (setup) and the global complex 5-point operator.
//
// Discretisation (Sec. 2, Eq. (pml); Sec. 3 "second order finite difference"):
// the operator J^{-1} div(A grad u) + k^2 u, A = diag(alpha2/alpha1,
// alpha1/alpha2), J = alpha1 alpha2, is multiplied by J h^2 and discretised in
// conservative form, giving the complex-symmetric row
//   west  alpha2(y_j) / alpha1(x_{i-1/2})     east  alpha2(y_j) / alpha1(x_{i+1/2})
//   south alpha1(x_i) / alpha2(y_{j-1/2})     north alpha1(x_i) / alpha2(y_{j+1/2})
//   centre -(sum of the four) + h^2 alpha1(x_i) alpha2(y_j) k^2(x_i, y_j)
// with zero (Dirichlet) values outside the box.  The same row builder serves
// the global operator and, in the factorisation, the local operators of
// Eq. (pmlij) with the box's own PML tables.
#include "hd_internal.cuh"

namespace hd {

// alpha = 1 + i s0 (xi / npml)^p at position `pos` (cell units) of a segment
// of `ncell` cells whose first and last `npml` cells are PML (Sec. 2: sigma = 0
// inside, > 0 in the layer; xi = distance into the layer).
__device__ __forceinline__ double2 pml_alpha(double pos, int ncell, int npml, double s0, int power) {
  if (npml <= 0) return make_double2(1.0, 0.0);
  double lo = (double)npml, hi = (double)(ncell - npml);
  double xi = pos < lo ? lo - pos : (pos > hi ? pos - hi : 0.0);
  double t = xi / (double)npml, p = 1.0;
  for (int e = 0; e < power; ++e) p *= t;
  return make_double2(1.0, s0 * p);
}

// Fills, for a segment of ncell cells: centre alphas a_c[ncell] and the
// reciprocals of the face alphas ia_f[ncell+1].
__device__ void fill_segment(double2 *a_c, double2 *ia_f, int ncell, int npml, double s0, int power, int t, int nt) {
  for (int l = t; l < ncell; l += nt) a_c[l] = pml_alpha(l + 0.5, ncell, npml, s0, power);
  for (int f = t; f <= ncell; f += nt) ia_f[f] = cinv(pml_alpha((double)f, ncell, npml, s0, power));
}

__global__ void k_global_tables(double2 *ax_c, double2 *iax_f, double2 *ay_c, double2 *iay_f, int NX, int NY,
                                int npml, double s0, int power) {
  int t = threadIdx.x, nt = blockDim.x;
  if (blockIdx.x == 0) fill_segment(ax_c, iax_f, NX, npml, s0, power, t, nt);
  else fill_segment(ay_c, iay_f, NY, npml, s0, power, t, nt);
}

// Per box: the PML of Omega_ij itself (its outer npml cells on every side).
__global__ void k_local_tables(const SubDev *subs, double2 *pool, int npml, double s0, int power) {
  const SubDev s = subs[blockIdx.x];
  double2 *a1c = pool + s.aoff;
  double2 *ia1f = a1c + s.ex;
  double2 *a2c = ia1f + s.ex + 1;
  double2 *ia2f = a2c + s.ey;
  fill_segment(a1c, ia1f, s.ex, npml, s0, power, threadIdx.x, blockDim.x);
  fill_segment(a2c, ia2f, s.ey, npml, s0, power, threadIdx.x, blockDim.x);
}

// k^2 = (omega / c)^2 per cell, and the centre coefficient h^2 k^2 - 4 that A has
// wherever both alphas are 1 (outside the PML).
__global__ void k_wavenumber(const double *__restrict__ c, double *__restrict__ k2, double *__restrict__ cc,
                             int64_t n, double omega, double h2, int32_t *status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ci = c[i];
  double k = omega / ci;
  if (!(ci > 0.0) || !isfinite(k)) atomicOr(status, ST_NONFINITE);
  const double kk = k * k;
  k2[i] = kk;
  cc[i] = add_rn(mul_rn(h2, kk), -4.0);
}

cudaError_t launch_setup_tables(hd_ctx *ctx, const double *c_dev, cudaStream_t st) {
  k_global_tables<<<2, 256, 0, st>>>(ctx->d_gax_c, ctx->d_giax_f, ctx->d_gay_c, ctx->d_giay_f, ctx->NX, ctx->NY,
                                     ctx->npml, ctx->s0, ctx->power);
  k_local_tables<<<ctx->nsub, 256, 0, st>>>(ctx->d_subs, ctx->d_lpool, ctx->npml, ctx->s0, ctx->power);
  int64_t n = (int64_t)ctx->NX * ctx->NY;
  k_wavenumber<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c_dev, ctx->d_k2, ctx->d_cc, n, ctx->omega,
                                                             ctx->h * ctx->h, ctx->d_status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- operator
struct OpArgs {
  const double2 *ax_c, *iax_f, *ay_c, *iay_f;
  const double *k2, *cc;
  int NX, NY, npml;
  double h2;
};

// y = A x on one grid per blockIdx.z; `mode` 0: y = A x, 1: y = b - A x.
template <int MODE>
__global__ void __launch_bounds__(256) k_stencil(OpArgs a, const double2 *__restrict__ x_all, int64_t xs_,
                                                 const double2 *__restrict__ b_all, int64_t bs_,
                                                 double2 *__restrict__ y_all, int64_t ys_) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= a.NX) return;
  const double2 *x = x_all + (int64_t)blockIdx.z * xs_;
  const double2 *b = MODE == 1 ? b_all + (int64_t)blockIdx.z * bs_ : nullptr;
  double2 *y = y_all + (int64_t)blockIdx.z * ys_;
  int64_t idx = (int64_t)j * a.NX + i;
  double2 xc = x[idx];
  double2 xw = i > 0 ? x[idx - 1] : make_double2(0.0, 0.0);
  double2 xe = i + 1 < a.NX ? x[idx + 1] : make_double2(0.0, 0.0);
  double2 xs = j > 0 ? x[idx - a.NX] : make_double2(0.0, 0.0);
  double2 xn = j + 1 < a.NY ? x[idx + a.NX] : make_double2(0.0, 0.0);
  double2 acc;
  if (i >= a.npml && i < a.NX - a.npml && j >= a.npml && j < a.NY - a.npml) {
    // outside the PML every alpha is 1: real coefficients 1, 1, 1, 1 and the stored
    // centre h^2 k^2 - 4 (8 FP64 operations per cell: the FP64 pipe bounds this kernel)
    const double cc = a.cc[idx];
    acc = make_double2(__fma_rn(cc, xc.x, xw.x), __fma_rn(cc, xc.y, xw.y));
    acc = make_double2(add_rn(acc.x, xe.x), add_rn(acc.y, xe.y));
    acc = make_double2(add_rn(acc.x, xs.x), add_rn(acc.y, xs.y));
    acc = make_double2(add_rn(acc.x, xn.x), add_rn(acc.y, xn.y));
  } else {
    double2 a1 = a.ax_c[i], a2 = a.ay_c[j];
    double2 cw = cmul(a2, a.iax_f[i]), ce = cmul(a2, a.iax_f[i + 1]);
    double2 cs = cmul(a1, a.iay_f[j]), cn = cmul(a1, a.iay_f[j + 1]);
    double2 j12 = cmul(a1, a2);
    double hk = mul_rn(a.h2, a.k2[idx]);
    double2 cc = make_double2(-(cw.x + ce.x + cs.x + cn.x) + hk * j12.x, -(cw.y + ce.y + cs.y + cn.y) + hk * j12.y);
    acc = cmul(cc, xc);
    acc = cfma(cw, xw, acc);
    acc = cfma(ce, xe, acc);
    acc = cfma(cs, xs, acc);
    acc = cfma(cn, xn, acc);
  }
  if (MODE == 1) acc = csub(b[idx], acc);
  y[idx] = acc;
}

static OpArgs op_args(hd_ctx *ctx) {
  OpArgs a;
  a.ax_c = ctx->d_gax_c; a.iax_f = ctx->d_giax_f; a.ay_c = ctx->d_gay_c; a.iay_f = ctx->d_giay_f;
  a.k2 = ctx->d_k2; a.cc = ctx->d_cc; a.NX = ctx->NX; a.NY = ctx->NY; a.npml = ctx->npml; a.h2 = ctx->h * ctx->h;
  return a;
}

cudaError_t launch_matvec(hd_ctx *ctx, const double2 *x, int64_t xs, double2 *y, int64_t ys, int nrhs,
                          cudaStream_t st) {
  dim3 grid((ctx->NX + 255) / 256, ctx->NY, nrhs);
  k_stencil<0><<<grid, 256, 0, st>>>(op_args(ctx), x, xs, nullptr, 0, y, ys);
  return cudaGetLastError();
}

cudaError_t launch_residual(hd_ctx *ctx, const double2 *b, const double2 *x, double2 *r, int nrhs, cudaStream_t st) {
  const int64_t n = (int64_t)ctx->NX * ctx->NY;
  dim3 grid((ctx->NX + 255) / 256, ctx->NY, nrhs);
  k_stencil<1><<<grid, 256, 0, st>>>(op_args(ctx), x, n, b, n, r, n);
  return cudaGetLastError();
}

cudaError_t launch_residual_strided(hd_ctx *ctx, const double2 *b, int64_t bs, const double2 *x, int64_t xs,
                                    double2 *r, int64_t rs, int nrhs, cudaStream_t st) {
  dim3 grid((ctx->NX + 255) / 256, ctx->NY, nrhs);
  k_stencil<1><<<grid, 256, 0, st>>>(op_args(ctx), x, xs, b, bs, r, rs);
  return cudaGetLastError();
}

__global__ void k_rhs(OpArgs a, const double2 *f, double2 *b) {  // b may alias f
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= a.NX) return;
  int64_t idx = (int64_t)j * a.NX + i;
  double2 jac = cmul(a.ax_c[i], a.ay_c[j]);
  double2 v = cmul(jac, f[idx]);
  b[idx] = make_double2(a.h2 * v.x, a.h2 * v.y);
}

cudaError_t launch_rhs(hd_ctx *ctx, const double2 *f, double2 *b, cudaStream_t st) {
  dim3 grid((ctx->NX + 255) / 256, ctx->NY);
  k_rhs<<<grid, 256, 0, st>>>(op_args(ctx), f, b);
  return cudaGetLastError();
}

}  // namespace hd
