"""Pins of the oracle's block flexible GMRES (many sources sharing one Krylov space),
checked against what the mathematics fixes rather than against itself:

* one right-hand side: the block method is FGMRES, so it must return the already
  pinned ``fgmres`` iterate step for step;
* the block Krylov space after k steps contains every column's own Krylov space, so
  each column's residual is no larger than that column's FGMRES residual after k
  steps with the same preconditioner (minimal residual over a larger space);
* to tolerance it is the dense solution, for a general matrix and for the Helmholtz
  operator with the DDM preconditioner; restarts keep that.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import DDMPreconditioner, Grid, block_fgmres, fgmres, global_operator, rhs_from_source


@pytest.fixture(scope="module")
def helmholtz():
    wl = W.make_workload("tiny", nb=4)
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c).tocsr()
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
    rng = np.random.default_rng(7)
    B = np.stack([rhs_from_source(g, W.gaussian_source(wl.N, wl.npml, *rng.uniform(0.2, 0.8, 2), 2.0 / wl.N)).ravel()
                  for _ in range(3)])
    return A, (lambda v: P.apply(v.reshape(g.n, g.n)).ravel()), B


def _res(A, B, X):
    return np.linalg.norm(B - (A @ X.T).T, axis=1) / np.linalg.norm(B, axis=1)


def test_one_column_is_fgmres(helmholtz):
    A, M, B = helmholtz
    for k in (1, 3, 6):
        s = fgmres(lambda v: A @ v, M, B[0], restart=10, rtol=1e-15, max_iters=k, reorth="always")
        blk = block_fgmres(lambda v: A @ v, M, B[:1], restart=10, rtol=1e-15, max_iters=k)
        assert s.iters == blk.iters == k
        assert np.linalg.norm(blk.x[0] - s.x) <= 1e-10 * np.linalg.norm(s.x)


@pytest.mark.parametrize("k", [2, 4])
def test_block_residual_bounded_by_each_columns_fgmres(helmholtz, k):
    A, M, B = helmholtz
    blk = block_fgmres(lambda v: A @ v, M, B, restart=10, rtol=1e-15, max_iters=k)
    rb = _res(A, B, blk.x)
    for c in range(B.shape[0]):
        s = fgmres(lambda v: A @ v, M, B[c], restart=10, rtol=1e-15, max_iters=k, reorth="always")
        rs = np.linalg.norm(B[c] - A @ s.x) / np.linalg.norm(B[c])
        assert rb[c] <= rs * (1 + 1e-8), (c, rb[c], rs)
    # and the estimates are the true residuals (orthonormal block basis)
    np.testing.assert_allclose(blk.relres_est, rb, rtol=1e-6)


def test_block_converges_to_dense_solution_general_matrix():
    rng = np.random.default_rng(3)
    n, p = 120, 3
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    B = rng.standard_normal((p, n)) + 1j * rng.standard_normal((p, n))
    res = block_fgmres(lambda v: A @ v, lambda v: v, B, restart=40, rtol=1e-12, max_iters=200)
    assert res.converged.all() and res.restarts == 1 and res.iters * p < n   # no exhaustion of the space
    np.testing.assert_allclose(res.x, np.linalg.solve(A, B.T).T, rtol=1e-10)


def test_block_space_exhaustion_ends_the_cycle_and_restarts():
    """With p k >= n the block Krylov space is the whole space: Gram-Schmidt cancels
    the new block to rounding, the cycle ends there, and the restart finishes the
    solve."""
    rng = np.random.default_rng(3)
    n, p = 40, 3
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    B = rng.standard_normal((p, n)) + 1j * rng.standard_normal((p, n))
    res = block_fgmres(lambda v: A @ v, lambda v: v, B, restart=n, rtol=1e-12, max_iters=200)
    assert res.converged.all() and res.restarts >= 1
    np.testing.assert_allclose(res.x, np.linalg.solve(A, B.T).T, rtol=1e-10)


def test_block_restarted_converges_with_the_ddm_preconditioner(helmholtz):
    A, M, B = helmholtz
    res = block_fgmres(lambda v: A @ v, M, B, restart=3, rtol=1e-9, max_iters=200)
    assert res.converged.all() and res.restarts >= 2
    assert (_res(A, B, res.x) <= 1e-9).all()
    xs = spla.spsolve(A.tocsc(), B[1])
    assert np.linalg.norm(res.x[1] - xs) / np.linalg.norm(xs) < 1e-6
