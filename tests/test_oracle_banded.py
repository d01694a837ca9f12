"""The oracle's own banded direct solver (oracle/banded_lu.c, banded Gaussian
elimination with partial pivoting) pinned against dense LAPACK solves, SuperLU
(a test-only cross-check) and the band structure it must respect."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import BandLU, DDMPreconditioner, Grid, box_order, decompose, local_operator


def _banded(n, kl, ku, rng, diag_scale=1.0):
    A = np.zeros((n, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        m = n - abs(d)
        A += np.diag(rng.standard_normal(m) + 1j * rng.standard_normal(m), d)
    A[np.arange(n), np.arange(n)] *= diag_scale
    return A


@pytest.mark.parametrize("n,kl,ku,scale", [(1, 0, 0, 1.0), (7, 2, 1, 1.0), (40, 3, 5, 1.0), (60, 5, 3, 1e-3),
                                           (50, 0, 4, 1.0), (50, 4, 0, 1.0), (33, 6, 6, 0.0)])
def test_band_lu_matches_dense_solve(n, kl, ku, scale):
    """Random banded matrices, also with a tiny or zero diagonal (so that partial
    pivoting must swap rows and the upper band fills to kl + ku): the backward error
    is at rounding level (partial pivoting is backward stable for these sizes) and the
    solution agrees with LAPACK's dense solve to cond(A) times rounding."""
    rng = np.random.default_rng(n * 100 + kl * 10 + ku)
    A = _banded(n, kl, ku, rng, scale)
    lu = BandLU(sp.csr_matrix(A))
    assert (lu.kl, lu.ku) == (kl if n > 1 else 0, ku if n > 1 else 0)
    cond = np.linalg.cond(A)
    for k in range(3):
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x = lu.solve(b)
        ref = np.linalg.solve(A, b)
        assert np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x)) < 1e-14
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-14 * cond + 1e-13
    if scale < 1e-2 and n > 1:
        assert np.any(lu.ipiv != np.arange(n)), "rows must have been swapped"


def test_band_lu_pivots_a_zero_diagonal_exactly():
    """A permutation matrix (every diagonal entry zero) inside the band is solved
    exactly: only row interchanges are needed."""
    n = 12
    P = np.zeros((n, n), dtype=np.complex128)
    for i in range(0, n, 2):
        P[i, i + 1] = 2.0 + 1j
        P[i + 1, i] = 1.0 - 3j
    b = np.arange(n) + 1j * np.arange(n)[::-1]
    x = BandLU(sp.csr_matrix(P)).solve(b)
    assert np.allclose(P @ x, b, rtol=0, atol=1e-14)


def test_band_lu_reports_a_singular_matrix():
    A = np.diag(np.ones(6, dtype=np.complex128))
    A[3, 3] = 0.0
    with pytest.raises(np.linalg.LinAlgError):
        BandLU(sp.csr_matrix(A))


def test_box_order_makes_the_band_the_short_side():
    """For a box wider than tall the unknowns are reordered y fastest, so the band of
    the local operator is its height; the solution is unchanged."""
    N, npml = 40, 6
    c = W.velocity_random_field(N, npml, seed=2)
    g = Grid(N, npml, 2 * np.pi * float(c.min()) * N / 10)
    k2 = (g.omega / c) ** 2
    subs = decompose(g, [6, 6 + 28, 46], [6, 46], overlap=3)   # 2 x 1 boxes: wider than tall
    s = subs[0]
    nx, ny = s.ex1 - s.ex0, s.ey1 - s.ey0
    assert nx != ny
    A = local_operator(g, k2, s)
    perm = box_order(nx, ny)
    lu = BandLU(A, perm)
    assert lu.kl == lu.ku == min(nx, ny)
    assert perm is None or sorted(perm.tolist()) == list(range(nx * ny))
    rng = np.random.default_rng(3)
    b = rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny)
    ref = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(lu.solve(b) - ref) / np.linalg.norm(ref) < 1e-11
    assert box_order(5, 7) is None and box_order(7, 5) is not None


def test_local_pml_solve_matches_dense_and_superlu():
    """The local PML problems of Eq. (pmlij) of a 2 x 2 decomposition: the oracle's
    banded LU agrees with the dense solve and with SuperLU (cross-check only)."""
    N, npml = 64, 8
    c = W.velocity_three_layer(N, npml)
    g = Grid(N, npml, 2 * np.pi * N / 10)
    k2 = (g.omega / c) ** 2
    rng = np.random.default_rng(5)
    for s in decompose(g, W.even_cuts(N, npml, 2), W.even_cuts(N, npml, 2), overlap=4):
        A = local_operator(g, k2, s)
        b = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
        x = BandLU(A, box_order(s.ex1 - s.ex0, s.ey1 - s.ey0)).solve(b)
        dense = np.linalg.solve(A.toarray(), b)
        slu = spla.splu(A.tocsc()).solve(b)
        assert np.linalg.norm(x - dense) / np.linalg.norm(dense) < 1e-11
        assert np.linalg.norm(x - slu) / np.linalg.norm(slu) < 1e-11
        # backward error at the level of FP64 rounding
        assert np.linalg.norm(A @ x - b) / (abs(A).max() * np.linalg.norm(x)) < 1e-13


def test_preconditioner_does_not_depend_on_thread_count():
    wl = W.make_workload("tiny")
    g = Grid(wl.N, wl.npml, wl.omega)
    r = W.random_complex((g.n, g.n), seed=9)
    z1 = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap, threads=1).apply(r)
    z4 = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap, threads=4).apply(r)
    assert np.array_equal(z1, z4)
