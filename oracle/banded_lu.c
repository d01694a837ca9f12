/*
 * Banded LU factorisation with partial pivoting and the matching solve, complex
 * FP64: the oracle's own direct solver of the local PML problems of Eq. (pmlij)
 * (Sec. 3 factorises each local problem once with a direct solver and does not
 * name it).  TEST INFRASTRUCTURE ONLY: loaded by the CPU oracle in this folder,
 * never by the CUDA library.
 *
 * This is textbook banded Gaussian elimination with row interchanges (Golub and
 * Van Loan, Matrix Computations, 4th ed., Sec. 4.3): a matrix with kl sub- and ku
 * superdiagonals keeps its lower bandwidth kl under partial pivoting while its
 * upper bandwidth grows to at most kl + ku.
 *
 * Storage (row-oriented band): row i of the n x n matrix occupies ld = 2 kl + ku + 1
 * complex entries starting at ab + 2 * i * ld (interleaved re, im); entry (i, j)
 * with -kl <= j - i <= kl + ku sits at position j - i + kl of that row.  Positions
 * beyond ku above the diagonal must be zero on input (room for the fill).  On
 * output the row holds U (j >= i) and the multipliers of L (j < i, as computed at
 * step j, before later interchanges), and ipiv[k] is the row swapped with row k at
 * step k.
 */
#include <math.h>
#include <stddef.h>

#define RE(i, j) ab[2 * ((size_t)(i) * ld + (size_t)((j) - (i) + kl))]
#define IM(i, j) ab[2 * ((size_t)(i) * ld + (size_t)((j) - (i) + kl)) + 1]

static int imin(int a, int b) { return a < b ? a : b; }

/* Returns 0, or k + 1 if the pivot of step k is exactly zero (the factorisation
 * stops there). */
int blu_factor(int n, int kl, int ku, double *ab, int *ipiv) {
  const int ld = 2 * kl + ku + 1;
  for (int k = 0; k < n; ++k) {
    const int last = imin(n - 1, k + kl);        /* rows that can hold column k */
    const int jend = imin(n - 1, k + kl + ku);   /* columns of row k after fill  */
    /* pivot: the largest |a(i, k)| over rows k .. last (first one on ties) */
    int p = k;
    double best = RE(k, k) * RE(k, k) + IM(k, k) * IM(k, k);
    for (int i = k + 1; i <= last; ++i) {
      const double v = RE(i, k) * RE(i, k) + IM(i, k) * IM(i, k);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    ipiv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k)
      for (int j = k; j <= jend; ++j) {
        const double tr = RE(k, j), ti = IM(k, j);
        RE(k, j) = RE(p, j);
        IM(k, j) = IM(p, j);
        RE(p, j) = tr;
        IM(p, j) = ti;
      }
    /* 1 / pivot */
    const double pr = RE(k, k), pi = IM(k, k);
    const double d = pr * pr + pi * pi;
    const double ir = pr / d, ii = -pi / d;
    for (int i = k + 1; i <= last; ++i) {
      /* multiplier l = a(i, k) / a(k, k), kept in place of a(i, k) */
      const double ar = RE(i, k), ai = IM(i, k);
      const double lr = ar * ir - ai * ii, li = ar * ii + ai * ir;
      RE(i, k) = lr;
      IM(i, k) = li;
      if (lr == 0.0 && li == 0.0) continue;
      /* row i -= l * row k over the columns right of k */
      for (int j = k + 1; j <= jend; ++j) {
        const double br = RE(k, j), bi = IM(k, j);
        RE(i, j) -= lr * br - li * bi;
        IM(i, j) -= lr * bi + li * br;
      }
    }
  }
  return 0;
}

/* Solves A x = b in place (b: n interleaved complex entries) with the output of
 * blu_factor: the interchanges and multipliers step by step, then U x = y
 * backwards. */
void blu_solve(int n, int kl, int ku, const double *ab, const int *ipiv, double *b) {
  const int ld = 2 * kl + ku + 1;
  for (int k = 0; k < n; ++k) {
    const int p = ipiv[k];
    if (p != k) {
      const double tr = b[2 * k], ti = b[2 * k + 1];
      b[2 * k] = b[2 * p];
      b[2 * k + 1] = b[2 * p + 1];
      b[2 * p] = tr;
      b[2 * p + 1] = ti;
    }
    const double yr = b[2 * k], yi = b[2 * k + 1];
    const int last = imin(n - 1, k + kl);
    for (int i = k + 1; i <= last; ++i) {
      const double lr = RE(i, k), li = IM(i, k);
      b[2 * i] -= lr * yr - li * yi;
      b[2 * i + 1] -= lr * yi + li * yr;
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double sr = b[2 * k], si = b[2 * k + 1];
    const int jend = imin(n - 1, k + kl + ku);
    for (int j = k + 1; j <= jend; ++j) {
      const double ur = RE(k, j), ui = IM(k, j);
      sr -= ur * b[2 * j] - ui * b[2 * j + 1];
      si -= ur * b[2 * j + 1] + ui * b[2 * j];
    }
    const double pr = RE(k, k), pi = IM(k, k);
    const double d = pr * pr + pi * pi;
    b[2 * k] = (sr * pr + si * pi) / d;
    b[2 * k + 1] = (si * pr - sr * pi) / d;
  }
}
