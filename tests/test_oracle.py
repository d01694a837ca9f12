"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the fact it checks; none re-types the oracle's own formula.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as ss

import workloads as W
from oracle import (DDMPreconditioner, Grid, decompose, fgmres, global_operator, local_operator,
                    pml_profile, rhs_from_source)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _solve(A, b):
    return spla.spsolve(A.tocsc(), b.ravel())


# ---------------------------------------------------------------- PML profile
def test_pml_profile_shape():
    """Sec. 2: sigma = 0 (alpha = 1 exactly) inside, Im(alpha) > 0 and growing in the layer,
    the same profile on both sides, and alpha = 1 + i s0 at the outer boundary face."""
    ac, af = pml_profile(40, 8, 20.0, 2)
    assert np.all(ac[8:32] == 1.0) and np.all(af[8:33] == 1.0)
    assert np.all(np.diff(ac[:8].imag) < 0) and np.all(ac[:8].imag > 0)
    np.testing.assert_array_equal(ac, ac[::-1])
    np.testing.assert_array_equal(af, af[::-1])
    assert af[0] == 1.0 + 20.0j
    assert np.all(ac.real == 1.0)


# ---------------------------------------------------------------- operator
def test_operator_complex_symmetric_not_hermitian():
    g = Grid(N=16, npml=4, omega=12.0)
    c = W.velocity_random_field(16, 4, seed=5)
    A = global_operator(g, c)
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 1e-3


def test_interior_rows_exact_on_cubics():
    """Away from the PML the rows are h^2 (Laplacian + k^2): the 5-point Laplacian
    is exact on cubic polynomials, so A u = h^2 (Delta u + k^2 u) there."""
    N, npml = 24, 6
    g = Grid(N=N, npml=npml, omega=7.0)
    c = W.velocity_three_layer(N, npml)
    k2 = (g.omega / c) ** 2
    x = W.cell_centres(N, npml)
    X, Y = np.meshgrid(x, x)
    u = 1.0 + 2 * X - Y + X * Y + 0.5 * X**3 - 2 * Y**2 * X + 0.25j * Y**3
    lap = 3.0 * X - 4.0 * X + 1.5j * Y        # closed-form Laplacian of u
    Au = (global_operator(g, c) @ u.ravel()).reshape(u.shape)
    ref = g.h**2 * (lap + k2 * u)
    s = slice(npml + 1, npml + N - 1)
    np.testing.assert_allclose(Au[s, s], ref[s, s], rtol=0, atol=1e-12)


def test_no_pml_gives_textbook_kronecker_sum():
    """With sigma = 0 the operator is the textbook Dirichlet 5-point matrix
    kron(I, T) + kron(T, I) + h^2 diag(k^2), T = tridiag(1, -2, 1)."""
    N, npml = 10, 3
    g = Grid(N=N, npml=npml, omega=9.0, sigma0_over_omega=0.0)
    c = W.velocity_random_field(N, npml, seed=3)
    n = g.n
    T = sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    ref = sp.kron(I, T) + sp.kron(T, I) + g.h**2 * sp.diags(((g.omega / c) ** 2).ravel())
    assert abs(global_operator(g, c) - ref).max() < 1e-14


def test_manufactured_solution_second_order():
    """A smooth compactly supported u* solves the PML problem exactly (f = 0 and
    u* = 0 in the layer), so the discrete error must fall 4x per grid halving."""
    k = 10.0

    def bump(t, a=0.2, L=0.6):
        th = np.pi * (t - a) / L
        inside = (t >= a) & (t <= a + L)
        s = np.sin(th)
        return (np.where(inside, s**6, 0.0),
                np.where(inside, (np.pi / L) ** 2 * (30 * s**4 * np.cos(th) ** 2 - 6 * s**6), 0.0))

    errs = []
    for N in (32, 64, 128):
        g = Grid(N=N, npml=8, omega=k)
        x = W.cell_centres(N, 8)
        b, b2 = bump(x)
        u = b[None, :] * b[:, None]
        f = b2[None, :] * b[:, None] + b[None, :] * b2[:, None] + k * k * u
        uh = _solve(global_operator(g, np.ones((g.n, g.n))), rhs_from_source(g, f)).reshape(g.n, g.n)
        errs.append(np.abs(uh - u).max() / np.abs(u).max())
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.7 < e0 / e1 < 4.3
    assert errs[-1] < 2e-3


def _hankel_error(N, s0=20.0, k=20.0, w=0.025):
    g = Grid(N=N, npml=16, omega=k, sigma0_over_omega=s0)
    x = W.cell_centres(N, 16)
    f = W.gaussian_source(N, 16, 0.5, 0.5, w)
    uh = _solve(global_operator(g, np.ones((g.n, g.n))), rhs_from_source(g, f)).reshape(g.n, g.n)
    r = np.hypot(x[None, :] - 0.5, x[:, None] - 0.5)
    # free-space outgoing field of a unit-mass Gaussian (Eq. (helm) with the
    # Sommerfeld condition): -(i/4) exp(-(k w)^2 / 2) H0^(1)(k r) for r >> w
    ue = -0.25j * math.exp(-(k * w) ** 2 / 2) * ss.hankel1(0, k * np.maximum(r, 1e-9))
    m = (r > 0.25) & (r < 0.45)
    return np.linalg.norm(uh[m] - ue[m]) / np.linalg.norm(ue[m])


def test_hankel_free_space_solution():
    """Homogeneous medium: the PML-truncated discrete field matches the free-space
    Hankel solution, with second-order convergence (PML reflection below it)."""
    e = [_hankel_error(N) for N in (64, 128, 256)]
    assert e[2] < 2.5e-3
    assert 3.5 < e[0] / e[1] < 4.6 and 3.5 < e[1] / e[2] < 4.6


def test_hankel_rejects_wrong_pml_sign():
    """Planted mistake: a PML with the opposite sign of sigma (incoming convention)
    must fail the same comparison by a wide margin."""
    assert _hankel_error(128, s0=-20.0) > 0.3


# ---------------------------------------------------------------- decomposition
def test_decomposition_matches_sec2_boxes():
    g = Grid(N=64, npml=8, omega=10.0)
    cuts = W.even_cuts(64, 8, 4)
    subs = decompose(g, cuts, cuts, overlap=3)
    s00, s10, s30 = subs[0], subs[1], subs[3]
    # x_{0,0} = x_0 - l_pml ; x_{i,0} = x_i - lo - l_pml ; x_{Nb-1,1} = x_Nb + l_pml
    assert (s00.ex0, s00.ex1) == (0, cuts[1] + 3 + 8)
    assert (s10.ex0, s10.ex1) == (cuts[1] - 3 - 8, cuts[2] + 3 + 8)
    assert (s30.ex0, s30.ex1) == (cuts[3] - 3 - 8, g.n)
    # owned boxes tile the whole grid (global-PML cells owned by boundary boxes)
    cover = np.zeros((g.n, g.n), int)
    for s in subs:
        cover[s.oy0:s.oy1, s.ox0:s.ox1] += 1
    assert np.all(cover == 1)
    lit = decompose(g, cuts, cuts, overlap=3, own_global_pml=False)
    cover[:] = 0
    for s in lit:
        cover[s.oy0:s.oy1, s.ox0:s.ox1] += 1
    assert cover.sum() == 64 * 64


# ---------------------------------------------------------------- preconditioner
def test_one_subdomain_is_exact_inverse():
    """Nb = 1: Omega_00 = Omega and its PML is the global PML, so M = A^{-1} and
    GMRES converges in exactly one iteration."""
    wl = W.make_workload("tiny", N=48, nb=1)
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c)
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
    r = W.random_complex(g.n * g.n, seed=11)
    np.testing.assert_allclose(P.apply(r).ravel(), _solve(A, r), rtol=1e-12, atol=1e-12)
    b = rhs_from_source(g, wl.f[0]).ravel()
    res = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, 20, 1e-10, 50)
    assert res.iters == 1 and res.converged and res.relres_true < 1e-12


def test_local_residual_vanishes_outside_local_pml():
    """Sec. 2: the local residual f_ij - L u_ij is zero inside Omega_ij away from
    its PML and non-zero in the local PML that faces the neighbours."""
    wl = W.make_workload("tiny", N=96, nb=3)
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c)
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap, subdomains=[4])
    s = P.subs[4]
    r = W.random_complex((g.n, g.n), seed=2)
    U = np.zeros((g.n, g.n), complex)
    U[s.ey0:s.ey1, s.ex0:s.ex1] = P.local_solve(4, r)
    chi = np.zeros_like(r)
    chi[s.oy0:s.oy1, s.ox0:s.ox1] = r[s.oy0:s.oy1, s.ox0:s.ox1]
    res = (A @ U.ravel()).reshape(g.n, g.n) - chi
    p = g.npml
    inner = res[s.ey0 + p:s.ey1 - p, s.ex0 + p:s.ex1 - p]
    assert np.abs(inner).max() < 1e-10 * np.abs(r).max()
    pml_band = res[s.ey0 + 1:s.ey0 + p, s.ex0 + p:s.ex1 - p]
    assert np.abs(pml_band).max() > 1e-3 * np.abs(r).max()


def test_dense_brute_force_preconditioner():
    """Eq. (pc) on a 12^2 grid with 2x2 boxes, formed densely: M = sum_ij E_ij^T
    inv(A_ij) X_ij with explicit 0/1 extension E and owned-restriction X."""
    N, npml = 12, 4
    g = Grid(N=N, npml=npml, omega=8.0)
    c = W.velocity_random_field(N, npml, seed=9)
    cuts = W.even_cuts(N, npml, 2)
    P = DDMPreconditioner(g, c, cuts, cuts, overlap=1)
    n2 = g.n * g.n
    M = np.zeros((n2, n2), complex)
    for s in P.subs:
        ex, ey = s.ex1 - s.ex0, s.ey1 - s.ey0
        E = np.zeros((ex * ey, n2))
        X = np.zeros((ex * ey, n2))
        for ly in range(ey):
            for lx in range(ex):
                gi = (s.ey0 + ly) * g.n + s.ex0 + lx
                E[ly * ex + lx, gi] = 1.0
                if s.ox0 <= s.ex0 + lx < s.ox1 and s.oy0 <= s.ey0 + ly < s.oy1:
                    X[ly * ex + lx, gi] = 1.0
        Ainv = np.linalg.inv(local_operator(g, P.k2, s).toarray())
        M += E.T @ Ainv @ X
    r = W.random_complex(n2, seed=4)
    np.testing.assert_allclose(P.apply(r).ravel(), M @ r, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- smoothing function (Remark after Eq. (pc))
def test_smoothstep_is_a_c2_step():
    """S(0) = 0, S(1) = 1 and S', S'' vanish at both ends (C^2 step), from the
    closed-form derivatives 30 t^2 (1 - t)^2 and 60 t (1 - t)(1 - 2 t)."""
    from oracle import smoothstep5
    t = np.linspace(0.0, 1.0, 2001)
    S = smoothstep5(t)
    assert S[0] == 0.0 and S[-1] == 1.0 and np.all(np.diff(S) >= 0)
    h = t[1] - t[0]
    d1 = np.gradient(S, h)
    d2 = np.gradient(d1, h)
    np.testing.assert_allclose(d1, 30 * t**2 * (1 - t)**2, atol=1e-4)
    np.testing.assert_allclose(d2[2:-2], (60 * t * (1 - t) * (1 - 2 * t))[2:-2], atol=1e-3)


def test_smoothing_profile_one_on_owned_zero_past_the_box():
    """beta = 1 on the owned cells, strictly between 0 and 1 in the band, and its
    continuation is 0 one cell past the box (the Remark: beta = 1 on the owned part,
    0 outside Omega_ij)."""
    from oracle import smoothing_profile, smoothstep5
    o0, o1, e0, e1 = 24, 88, 12, 100
    b = smoothing_profile(o0, o1, e0, e1)
    assert np.all(b[o0 - e0:o1 - e0] == 1.0)
    band = np.r_[b[:o0 - e0], b[o1 - e0:]]
    assert np.all((band > 0) & (band < 1))
    assert smoothstep5(1.0 - (o0 - (e0 - 1)) / (o0 - e0 + 1.0)) == 0.0
    assert np.all(np.diff(b[:o0 - e0 + 1]) > 0) and np.all(np.diff(b[o1 - e0 - 1:]) < 0)


def test_smoothed_preconditioner_dense_brute_force():
    """sum_ij E_ij^T diag(beta_ij) inv(A_ij) X_ij formed densely on 12^2 with 2x2 boxes
    equals the smoothed application; with one box beta is 1 on the whole box and
    the smoothed preconditioner is still the exact inverse."""
    N, npml = 12, 4
    g = Grid(N=N, npml=npml, omega=8.0)
    c = W.velocity_random_field(N, npml, seed=9)
    cuts = W.even_cuts(N, npml, 2)
    P = DDMPreconditioner(g, c, cuts, cuts, overlap=1, smoothing=True)
    n2 = g.n * g.n
    M = np.zeros((n2, n2), complex)
    for b, s in enumerate(P.subs):
        ex, ey = s.ex1 - s.ex0, s.ey1 - s.ey0
        E = np.zeros((ex * ey, n2))
        X = np.zeros((ex * ey, n2))
        for ly in range(ey):
            for lx in range(ex):
                gi = (s.ey0 + ly) * g.n + s.ex0 + lx
                E[ly * ex + lx, gi] = 1.0
                if s.ox0 <= s.ex0 + lx < s.ox1 and s.oy0 <= s.ey0 + ly < s.oy1:
                    X[ly * ex + lx, gi] = 1.0
        Ainv = np.linalg.inv(local_operator(g, P.k2, s).toarray())
        M += E.T @ np.diag(P.beta(b).ravel()) @ Ainv @ X
    r = W.random_complex(n2, seed=4)
    np.testing.assert_allclose(P.apply(r).ravel(), M @ r, rtol=1e-11, atol=1e-12)
    assert not np.allclose(P.apply(r), DDMPreconditioner(g, c, cuts, cuts, overlap=1).apply(r))
    wl = W.make_workload("tiny", N=48, nb=1)
    g1 = Grid(wl.N, wl.npml, wl.omega)
    P1 = DDMPreconditioner(g1, wl.c, wl.cut_x, wl.cut_y, wl.overlap, smoothing=True)
    r1 = W.random_complex(g1.n * g1.n, seed=11)
    np.testing.assert_allclose(P1.apply(r1).ravel(), _solve(global_operator(g1, wl.c), r1), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- multi-step DDM
def _ddm_case():
    wl = W.make_workload("tiny", N=96, nb=3, medium="three_layer")
    g = Grid(wl.N, wl.npml, wl.omega)
    return wl, g, global_operator(g, wl.c), DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)


def test_multistep_equals_residual_correction():
    """Eq. (ddms) with the Sec. 2 fact that a box's own residual vanishes on its
    owned part: the step-(s+1) sources are exactly the global residual f - A z_s of
    the sum so far, restricted to the owned boxes, so s steps of Eq. (ddms) + (sum)
    equal z_{s+1} = z_s + M (f - A z_s), z_0 = M f (M: Eq. (pc)).  A dropped corner
    neighbour, a wrong sign or a wrong restriction breaks this."""
    wl, g, A, P = _ddm_case()
    f = W.random_complex((g.n, g.n), seed=21)
    z = P.apply(f)
    for steps in (1, 2, 3):
        if steps > 1:
            z = z + P.apply((f.ravel() - A @ z.ravel()).reshape(g.n, g.n))
        zs = P.apply_multistep(f, steps)
        assert np.linalg.norm(zs - z) / np.linalg.norm(z) < 1e-12


def test_multistep_solver_converges():
    """Sec. 2: the iteration goes on until the residual is small; each step carries
    the waves one more box, so the residual of the DDM sum falls with the steps."""
    wl, g, A, P = _ddm_case()
    b = rhs_from_source(g, wl.f[0])
    res = [np.linalg.norm(b.ravel() - A @ P.apply_multistep(b, k).ravel()) / np.linalg.norm(b) for k in (1, 3, 6)]
    assert res[1] < 0.5 * res[0] and res[2] < 0.2 * res[0]


def test_multistep_one_box_adds_nothing():
    """With one box there are no neighbours: every step after the first has zero
    sources, and the sum is the exact solve of the one-box case."""
    wl = W.make_workload("tiny", N=48, nb=1)
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c)
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
    r = W.random_complex((g.n, g.n), seed=13)
    np.testing.assert_allclose(P.apply_multistep(r, 3).ravel(), _solve(A, r.ravel()), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- GMRES
def test_fgmres_identity_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 40
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    res = fgmres(lambda v: A @ v, lambda v: v, b, restart=n, rtol=1e-13, max_iters=200)
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), rtol=1e-11)
    assert res.converged and res.iters <= n
    assert abs(res.relres_est - res.relres_true) < 1e-12


@pytest.mark.parametrize("reorth", ["always", "selective"])
def test_fgmres_reorth_modes_match_dense_solve(reorth):
    """Both Gram-Schmidt variants solve a system whose Krylov vectors become nearly
    dependent (eigenvalues spread over four decades), where one classical pass alone
    loses orthogonality; the selective rule must still reach the dense solution."""
    rng = np.random.default_rng(5)
    n = 48
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    A = (Q * np.logspace(0, 4, n)) @ Q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    res = fgmres(lambda v: A @ v, lambda v: v, b, restart=n, rtol=1e-11, max_iters=4 * n, reorth=reorth)
    assert res.converged and res.iters <= n
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-9   # cond(A) = 1e4
    assert np.linalg.norm(b - A @ res.x) / np.linalg.norm(b) <= 1e-11


def test_fgmres_restarted_converges():
    rng = np.random.default_rng(1)
    n = 60
    A = np.diag(np.linspace(1, 3, n)) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    res = fgmres(lambda v: A @ v, lambda v: v, b, restart=5, rtol=1e-10, max_iters=500)
    assert res.converged and res.restarts > 1
    assert np.linalg.norm(b - A @ res.x) / np.linalg.norm(b) <= 1e-10


def test_iterations_grow_with_subdomains_per_direction():
    """Abstract and Sec. 3.1 (Table 2): with the subdomain size fixed the
    iteration count grows in proportion to Nb; the paper's growth per doubling of
    Nb is 2.0-2.6."""
    with open(os.path.join(GOLDEN, "paper_table2_const_weak.json")) as fh:
        paper = json.load(fh)
    pr = np.array(paper["iterations"][1:4]) / np.array(paper["iterations"][0:3])
    assert np.all((pr > 1.9) & (pr < 2.7))
    its = []
    for nb in (2, 4, 8):
        wl = W.make_workload("tiny", N=32 * nb, nb=nb)
        g = Grid(wl.N, wl.npml, wl.omega)
        A = global_operator(g, wl.c)
        P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
        b = rhs_from_source(g, wl.f[0]).ravel()
        res = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, 50, 1e-8, 400)
        assert res.converged
        its.append(res.iters)
    ratios = np.array(its[1:]) / np.array(its[:-1])
    assert np.all((ratios > 1.5) & (ratios < 3.2)), its


def test_tiny_config_converges_fast():
    """Tiny configuration (128^2, 2x2 boxes): a handful of iterations, relres 1e-8."""
    wl = W.make_workload("tiny")
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c)
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
    b = rhs_from_source(g, wl.f[0]).ravel()
    res = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, wl.restart, wl.rtol, 200)
    assert res.converged and res.iters <= 12
    assert np.linalg.norm(b - A @ res.x) / np.linalg.norm(b) <= wl.rtol
