"""The lazily normalised Arnoldi recurrence of the double-single Gram-Schmidt mode,
checked on the CPU against the normalised one (Sec. 3's FGMRES with CGS2).

The GPU stores each new basis vector unnormalised: u_0 = v_0, then per step
w = A M u_j, h1_k = u_k^H w, y = g (w - sum_k sc_k^2 h1_k u_k) with g = 1/||w||, an
optional second pass h2_k = u_k^H y, y -= sum_k sc_k^2 h2_k u_k, and sc_{j+1} = 1/||y||;
the Hessenberg entries are h_kj = sc_j sc_k (h1_k + h2_k / g), h_{j+1,j} = sc_j ||y|| / g,
and the solution takes sc_j eta_j with the stored z'_j = M u_j.  Written out here in
numpy over the oracle's operator and preconditioner, it must give the same Hessenberg
matrix and the same FGMRES iterate as normalising every vector, and keep every stored
norm in (0, 1].
"""
import numpy as np
import pytest

import workloads as W
from oracle import DDMPreconditioner, Grid, global_operator, rhs_from_source

R = 8


@pytest.fixture(scope="module")
def problem():
    wl = W.make_workload("tiny", nb=4)   # 4x4 boxes: no near-breakdown within R steps
    g = Grid(wl.N, wl.npml, wl.omega)
    A = global_operator(g, wl.c)
    P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap)
    b = rhs_from_source(g, wl.f[0]).ravel()
    return A, (lambda v: P.apply(v.reshape(g.n, g.n)).ravel()), b


def _second_pass(mode, left2, w2):
    return mode == "always" or left2 < 0.01 * w2


def _normalised(A, M, b, mode):
    V, Z = [b / np.linalg.norm(b)], []
    H = np.zeros((R + 1, R), complex)
    for j in range(R):
        Z.append(M(V[j]))
        w = A @ Z[j]
        w2 = np.vdot(w, w).real
        h = np.array([v.conj() @ w for v in V])
        w = w - sum(c * v for c, v in zip(h, V))
        if _second_pass(mode, np.vdot(w, w).real, w2):
            h2 = np.array([v.conj() @ w for v in V])
            w = w - sum(c * v for c, v in zip(h2, V))
            h = h + h2
        hn = np.linalg.norm(w)
        H[:j + 1, j], H[j + 1, j] = h, hn
        V.append(w / hn)
    return H, Z, [1.0] * R


def _lazy(A, M, b, mode):
    U, Z, sc = [b / np.linalg.norm(b)], [], [1.0]
    H = np.zeros((R + 1, R), complex)
    norms = []
    for j in range(R):
        Z.append(M(U[j]))
        w = A @ Z[j]
        h1 = np.array([u.conj() @ w for u in U])
        w2 = np.vdot(w, w).real
        g = 1.0 / np.sqrt(w2)
        y = g * w - sum(g * sc[k] ** 2 * h1[k] * U[k] for k in range(j + 1))
        h2 = np.zeros(j + 1, complex)
        if _second_pass(mode, np.vdot(y, y).real / g ** 2, w2):
            h2 = np.array([u.conj() @ y for u in U])
            y = y - sum(sc[k] ** 2 * h2[k] * U[k] for k in range(j + 1))
        yn = np.linalg.norm(y)
        H[:j + 1, j] = sc[j] * np.asarray(sc[:j + 1]) * (h1 + h2 / g)
        H[j + 1, j] = sc[j] * yn / g
        sc.append(1.0 / yn)
        U.append(y)
        norms.append(yn)
    return H, Z, sc[:R], norms


@pytest.mark.parametrize("mode", ["selective", "always"])
def test_lazy_recurrence_matches_normalised(problem, mode):
    A, M, b = problem
    Hn, Zn, sn = _normalised(A, M, b, mode)
    Hl, Zl, sl, norms = _lazy(A, M, b, mode)
    assert np.linalg.norm(Hl - Hn) <= 1e-10 * np.linalg.norm(Hn)
    e1 = np.zeros(R + 1, complex)
    e1[0] = np.linalg.norm(b)
    xn = sum(z * c * s for z, c, s in zip(Zn, np.linalg.lstsq(Hn, e1, rcond=None)[0], sn))
    xl = sum(z * c * s for z, c, s in zip(Zl, np.linalg.lstsq(Hl, e1, rcond=None)[0], sl))
    assert np.linalg.norm(xl - xn) <= 1e-12 * np.linalg.norm(xn)
    assert all(0.0 < q <= 1.0 + 1e-12 for q in norms)     # g keeps every stored norm in (0, 1]


def test_lazy_recurrence_catches_a_missing_scale(problem):
    """Dropping g from h_{j+1,j} (a plausible slip) breaks the agreement."""
    A, M, b = problem
    Hn, _, _ = _normalised(A, M, b, "selective")
    Hl, _, sc, norms = _lazy(A, M, b, "selective")
    bad = Hl.copy()
    for j in range(R):
        bad[j + 1, j] = (1.0 if j == 0 else 1.0 / norms[j - 1]) * norms[j]   # sc_j ||y|| without / g
    assert np.linalg.norm(bad - Hn) > 1e-3 * np.linalg.norm(Hn)
