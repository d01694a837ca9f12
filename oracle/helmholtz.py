"""FP64 CPU oracle: PML Helmholtz operator, overlapping decomposition, one-step
DDM preconditioner and FGMRES, written step by step from the paper
(Leng & Ju, "An overlapping domain decomposition preconditioner for the
Helmholtz equation", arXiv 1508.02897).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU baseline
of the benchmark, never by the product path.  It shares no code with the CUDA
path; only the seeded input generators in ``workloads`` serve both.

Every function cites the passage it follows.  Where the paper is silent or
garbled the reading used is stated in the docstring:

* Grid: cell-centred, interior [0,1]^2 of N x N cells, npml cells of PML on
  every side, homogeneous Dirichlet just outside the truncated domain (Sec. 2
  defines Omega; the paper prints no grid).
* PML: alpha_j(t) = 1 + i sigma_j(t)/omega with sigma(xi) = s0*omega*(xi/l_pml)^p,
  xi the distance into the layer (Sec. 2, Eq. (pml): the paper names alpha
  without defining it; the +i sign makes e^{ikr}, the outgoing wave of the
  Sommerfeld condition in Eq. (helm), decay in the layer).
* Stencil: conservative 5-point form of J^{-1} div(A grad u) + k^2 u multiplied
  by J h^2, which makes the matrix complex symmetric (Sec. 3 says only
  "second order finite difference").
* Ownership: boundary subdomains also own the adjacent global-PML cells, so the
  owned boxes tile the whole grid (Sec. 2 defines the owned boxes on the
  interior only; ``own_global_pml=False`` gives the literal reading).
* Krylov: right-preconditioned flexible GMRES (Z_j = M v_j stored), x0 = 0,
  classical Gram-Schmidt applied twice, complex Givens rotations with real
  cosine, stop when |g_{j+1}| <= rtol ||b|| and the true residual agrees
  (Sec. 3 says "GMRES" with a restart and a relative tolerance).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

from .banded import BandLU, box_order

__all__ = [
    "Grid", "Subdomain", "pml_profile", "helmholtz_matrix", "global_operator", "rhs_from_source",
    "decompose", "local_operator", "factor_box", "oracle_threads", "DDMPreconditioner", "fgmres", "FGMRESResult",
    "smoothstep5", "smoothing_profile",
]


@dataclass
class Grid:
    """Truncated domain Omega of Sec. 2: N x N interior cells of width h = 1/N plus npml PML cells per side."""
    N: int
    npml: int
    omega: float
    sigma0_over_omega: float = 20.0
    pml_power: int = 2

    @property
    def n(self) -> int:
        return self.N + 2 * self.npml

    @property
    def h(self) -> float:
        return 1.0 / self.N


def pml_profile(ncell: int, npml: int, s0: float, power: int):
    """Stretching factors alpha = 1 + i sigma/omega along one axis of a segment of
    ``ncell`` cells whose first and last ``npml`` cells form the PML (Sec. 2,
    uniaxial PML; sigma = 0 inside, > 0 in the layer).

    sigma(xi)/omega = s0 (xi / l_pml)^power with l_pml = npml h; the cell width
    cancels, so xi is measured in cells.  Returns (alpha at the ncell cell
    centres, alpha at the ncell+1 faces; face f lies between cells f-1 and f).
    """
    def alpha(xi):
        return 1.0 + 1j * s0 * (np.asarray(xi, dtype=np.float64) / npml) ** power

    c = np.arange(ncell, dtype=np.float64) + 0.5          # centre positions in cell units
    f = np.arange(ncell + 1, dtype=np.float64)            # face positions
    lo, hi = float(npml), float(ncell - npml)             # inner PML interfaces
    xi_c = np.where(c < lo, lo - c, np.where(c > hi, c - hi, 0.0))
    xi_f = np.where(f < lo, lo - f, np.where(f > hi, f - hi, 0.0))
    if npml == 0:
        return np.ones(ncell, np.complex128), np.ones(ncell + 1, np.complex128)
    return alpha(xi_c), alpha(xi_f)


def helmholtz_matrix(k2: np.ndarray, ax_c, ax_f, ay_c, ay_f, h: float) -> sp.csr_matrix:
    """Discrete PML operator of Eq. (pml), J^{-1} div(A grad u) + k^2 u with
    A = diag(alpha2/alpha1, alpha1/alpha2) and J = alpha1 alpha2, multiplied by
    J h^2.  Unknown (x=i, y=j) has index j*nx + i; Dirichlet outside the box.

    Row (i, j):  west/east  alpha2(y_j)/alpha1(x_{i-+1/2}),
                 south/north alpha1(x_i)/alpha2(y_{j-+1/2}),
                 centre -(sum of the four) + h^2 alpha1(x_i) alpha2(y_j) k2[j, i].
    """
    ny, nx = k2.shape
    ax_c = np.asarray(ax_c); ax_f = np.asarray(ax_f); ay_c = np.asarray(ay_c); ay_f = np.asarray(ay_f)
    w_w = ay_c[:, None] / ax_f[None, :-1]            # [ny][nx] coefficient of u(i-1, j)
    w_e = ay_c[:, None] / ax_f[None, 1:]             # u(i+1, j)
    w_s = ax_c[None, :] / ay_f[:-1, None]            # u(i, j-1)
    w_n = ax_c[None, :] / ay_f[1:, None]             # u(i, j+1)
    w_c = -(w_w + w_e + w_s + w_n) + h * h * ay_c[:, None] * ax_c[None, :] * k2
    idx = np.arange(nx * ny).reshape(ny, nx)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [w_c.ravel()]
    for wt, di, dj in ((w_w, -1, 0), (w_e, 1, 0), (w_s, 0, -1), (w_n, 0, 1)):
        jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ok = (ii + di >= 0) & (ii + di < nx) & (jj + dj >= 0) & (jj + dj < ny)
        rows.append(idx[ok]); cols.append(idx[(jj + dj)[ok], (ii + di)[ok]]); vals.append(wt[ok])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny))
    return A.tocsr()


def global_operator(grid: Grid, c: np.ndarray) -> sp.csr_matrix:
    """Operator of Eq. (pml) on the whole truncated domain Omega with k = omega / c."""
    k2 = (grid.omega / np.asarray(c, dtype=np.float64)) ** 2
    ax_c, ax_f = pml_profile(grid.n, grid.npml, grid.sigma0_over_omega, grid.pml_power)
    return helmholtz_matrix(k2, ax_c, ax_f, ax_c, ax_f, grid.h)


def rhs_from_source(grid: Grid, f: np.ndarray) -> np.ndarray:
    """Right-hand side J h^2 f of the scaled system (the same scaling as the rows)."""
    ax_c, _ = pml_profile(grid.n, grid.npml, grid.sigma0_over_omega, grid.pml_power)
    J = ax_c[:, None] * ax_c[None, :]
    return (grid.h * grid.h) * J * np.asarray(f, dtype=np.complex128)


@dataclass
class Subdomain:
    """Owned box [ox0,ox1) x [oy0,oy1) (the tilde-Omega_ij of Sec. 2) and the
    overlapping box [ex0,ex1) x [ey0,ey1) (Omega_ij), in global cell indices."""
    i: int
    j: int
    ox0: int
    ox1: int
    oy0: int
    oy1: int
    ex0: int
    ex1: int
    ey0: int
    ey1: int


def _ranges(cuts: Sequence[int], n: int, npml: int, overlap: int, own_global_pml: bool):
    nb = len(cuts) - 1
    out = []
    for i in range(nb):
        o0, o1 = cuts[i], cuts[i + 1]
        # Sec. 2: x_{i,0} = x_i - l_pml for i = 0, x_i - lo - l_pml otherwise;
        #         x_{i,1} = x_{i+1} + l_pml for the last box, x_{i+1} + lo + l_pml otherwise.
        e0 = o0 - npml - (overlap if i > 0 else 0)
        e1 = o1 + npml + (overlap if i < nb - 1 else 0)
        if own_global_pml:
            if i == 0:
                o0 = 0
            if i == nb - 1:
                o1 = n
        out.append((o0, o1, e0, e1))
    return out


def decompose(grid: Grid, cut_x: Sequence[int], cut_y: Sequence[int], overlap: int,
              own_global_pml: bool = True) -> List[Subdomain]:
    """Nb_x x Nb_y owned boxes and their overlapping extensions (Sec. 2, Fig. 1).

    ``cut_x``/``cut_y`` are interior cut points npml = c_0 < ... < c_Nb = npml + N
    (the x_i, y_j of Sec. 2; uneven cuts allowed).
    """
    n = grid.n
    rx = _ranges(cut_x, n, grid.npml, overlap, own_global_pml)
    ry = _ranges(cut_y, n, grid.npml, overlap, own_global_pml)
    subs = []
    for j, (oy0, oy1, ey0, ey1) in enumerate(ry):
        for i, (ox0, ox1, ex0, ex1) in enumerate(rx):
            assert 0 <= ex0 and ex1 <= n, "overlapping box leaves the truncated domain"
            subs.append(Subdomain(i, j, ox0, ox1, oy0, oy1, ex0, ex1, ey0, ey1))
    return subs


def local_operator(grid: Grid, k2: np.ndarray, s: Subdomain) -> sp.csr_matrix:
    """Local PML problem of Eq. (pmlij) on Omega_ij: the same operator with the
    PML of Omega_ij itself (its outer npml cells on every side) and the global k^2
    restricted to the box; Dirichlet outside the box."""
    ex, ey = s.ex1 - s.ex0, s.ey1 - s.ey0
    ax_c, ax_f = pml_profile(ex, grid.npml, grid.sigma0_over_omega, grid.pml_power)
    ay_c, ay_f = pml_profile(ey, grid.npml, grid.sigma0_over_omega, grid.pml_power)
    return helmholtz_matrix(k2[s.ey0:s.ey1, s.ex0:s.ex1], ax_c, ax_f, ay_c, ay_f, grid.h)


def smoothstep5(t: np.ndarray) -> np.ndarray:
    """t^3 (10 - 15 t + 6 t^2): 0 at t = 0, 1 at t = 1, first and second derivatives
    zero at both ends (a C^2 step)."""
    t = np.clip(np.asarray(t, dtype=np.float64), 0.0, 1.0)
    return t * t * t * (10.0 - 15.0 * t + 6.0 * t * t)


def smoothing_profile(o0: int, o1: int, e0: int, e1: int) -> np.ndarray:
    """One axis of the smoothing function beta_ij of the Remark after Eq. (pc) over the
    cells [e0, e1) of a box: 1 on the owned cells [o0, o1), falling to 0 across the band
    between the owned part and the edge of the box (reading: beta is the tensor product
    of C^2 steps of the cell distance d from the owned part, beta = S(1 - d / (W + 1))
    with W the band width, so it reaches 0 just outside the box)."""
    x = np.arange(e0, e1)
    b = np.ones(e1 - e0)
    lo = x < o0
    b[lo] = smoothstep5(1.0 - (o0 - x[lo]) / (o0 - e0 + 1.0))
    hi = x >= o1
    b[hi] = smoothstep5(1.0 - (x[hi] - o1 + 1) / (e1 - o1 + 1.0))
    return b


def factor_box(grid: Grid, k2: np.ndarray, s: Subdomain) -> BandLU:
    """The local PML problem of Eq. (pmlij) on box s, factorised once with the
    oracle's own banded LU with partial pivoting (Sec. 3: "factorized and solved
    with direct solver"; the paper does not name it), unknowns ordered so that the
    band is the shorter side of the box (bandwidth min(width, height))."""
    return BandLU(local_operator(grid, k2, s), box_order(s.ex1 - s.ex0, s.ey1 - s.ey0))


def oracle_threads() -> int:
    """Threads that factorise or solve boxes at once: HD_ORACLE_THREADS, else every host core."""
    return max(1, int(os.environ.get("HD_ORACLE_THREADS", "0")) or (os.cpu_count() or 1))


_pools = {}


def _pool(n: int) -> ThreadPoolExecutor:
    """A process-wide thread pool of n workers (the banded solver releases the GIL)."""
    if n not in _pools:
        _pools[n] = ThreadPoolExecutor(max_workers=n)
    return _pools[n]


class DDMPreconditioner:
    """One-step preconditioner of Eq. (ddm0) and Eq. (pc): restrict the input to
    every owned box, solve every local PML problem, and add each full local
    solution (including its PML area) into the output.  No smoothing function
    (the Remark after Eq. (pc) omits it).  Each local problem is factorised once
    with the oracle's banded direct solver (``factor_box``); the boxes are
    independent, so several factorise at once in threads (``threads``, default
    ``oracle_threads()``); the result does not depend on the thread count."""

    def __init__(self, grid: Grid, c: np.ndarray, cut_x, cut_y, overlap: int,
                 own_global_pml: bool = True, subdomains: Optional[Sequence[int]] = None, smoothing: bool = False,
                 threads: Optional[int] = None):
        self.grid = grid
        self.smoothing = smoothing
        self.c = np.asarray(c, dtype=np.float64)
        self.k2 = (grid.omega / self.c) ** 2
        self._A = None
        self.subs = decompose(grid, cut_x, cut_y, overlap, own_global_pml)
        self.active = list(range(len(self.subs))) if subdomains is None else list(subdomains)
        self.threads = min(threads or oracle_threads(), max(1, len(self.active)))
        lus = list(_pool(self.threads).map(lambda t: factor_box(grid, self.k2, self.subs[t]), self.active))
        self.lu = dict(zip(self.active, lus))

    def local_solve(self, s_idx: int, r: np.ndarray) -> np.ndarray:
        """u_ij^0 of Eq. (ddm0): local solve with r restricted to the owned box."""
        s = self.subs[s_idx]
        rho = np.zeros((s.ey1 - s.ey0, s.ex1 - s.ex0), dtype=np.complex128)
        rho[s.oy0 - s.ey0:s.oy1 - s.ey0, s.ox0 - s.ex0:s.ox1 - s.ex0] = r[s.oy0:s.oy1, s.ox0:s.ox1]
        return self.lu[s_idx].solve(rho.ravel()).reshape(rho.shape)

    def beta(self, s_idx: int) -> np.ndarray:
        """beta_ij over the box (rows y, columns x), Remark after Eq. (pc)."""
        s = self.subs[s_idx]
        return np.outer(smoothing_profile(s.oy0, s.oy1, s.ey0, s.ey1), smoothing_profile(s.ox0, s.ox1, s.ex0, s.ex1))

    def apply(self, r: np.ndarray) -> np.ndarray:
        """u_PC = sum_ij u_ij^0 over each full box Omega_ij, Eq. (pc); with smoothing,
        sum_ij beta_ij u_ij^0 (the Remark after Eq. (pc))."""
        r = np.asarray(r, dtype=np.complex128).reshape(self.grid.n, self.grid.n)
        z = np.zeros_like(r)
        # the local solves are independent (threads); the sum runs in box order
        sols = list(_pool(self.threads).map(lambda t: self.local_solve(t, r), self.active))
        for s_idx, u in zip(self.active, sols):
            s = self.subs[s_idx]
            z[s.ey0:s.ey1, s.ex0:s.ex1] += self.beta(s_idx) * u if self.smoothing else u
        return z

    def neighbours(self, s_idx: int) -> List[int]:
        """The index set N_ij of Sec. 2: the (up to 8) boxes whose i, j differ by at most 1."""
        s = self.subs[s_idx]
        return [t for t in self.active if t != s_idx
                and abs(self.subs[t].i - s.i) <= 1 and abs(self.subs[t].j - s.j) <= 1]

    def apply_multistep(self, f: np.ndarray, steps: int) -> np.ndarray:
        """The overlapping DDM of Eq. (ddm0), (ddms) and (sum), run for ``steps``
        steps (steps = 1 is the one-step preconditioner of Eq. (pc)).

        Step 0 solves every box with f restricted to its owned box.  Step s+1
        solves box ij with minus the sum over its neighbours N_ij of L applied to
        their step-s solutions (each extended by zero outside its box), restricted
        to the owned box of ij; L is the operator of the whole truncated domain.
        The result is the sum of every step's local solutions over their full boxes.
        """
        if steps < 1:
            raise ValueError("steps must be >= 1")
        if self.smoothing:
            raise ValueError("the multi-step form is built without the smoothing function")
        g = self.grid
        if self._A is None:
            self._A = global_operator(g, self.c)
        f = np.asarray(f, dtype=np.complex128).reshape(g.n, g.n)
        z = np.zeros_like(f)
        u = {}
        for s_idx in self.active:
            s = self.subs[s_idx]
            u[s_idx] = self.local_solve(s_idx, f)
            z[s.ey0:s.ey1, s.ex0:s.ex1] += u[s_idx]
        for _ in range(1, steps):
            Lu = {}
            for t in self.active:                       # L(u_t^s), u_t^s extended by zero
                st = self.subs[t]
                e = np.zeros_like(f)
                e[st.ey0:st.ey1, st.ex0:st.ex1] = u[t]
                Lu[t] = (self._A @ e.ravel()).reshape(g.n, g.n)
            u_next = {}
            for s_idx in self.active:
                src = np.zeros_like(f)
                for t in self.neighbours(s_idx):
                    src -= Lu[t]
                s = self.subs[s_idx]
                u_next[s_idx] = self.local_solve(s_idx, src)    # restricted to the owned box
                z[s.ey0:s.ey1, s.ex0:s.ex1] += u_next[s_idx]
            u = u_next
        return z


@dataclass
class FGMRESResult:
    x: np.ndarray
    iters: int
    restarts: int
    converged: bool
    relres_est: float
    relres_true: float
    history: List[float] = field(default_factory=list)


def _givens(a: complex, b: complex):
    """Rotation [c s; -conj(s) c] with real c that maps (a, b) to (gamma, 0)."""
    aa, bb = abs(a), abs(b)
    if bb == 0.0:
        return 1.0, 0.0 + 0.0j
    if aa == 0.0:
        return 0.0, complex(np.conj(b) / bb)
    t = math.hypot(aa, bb)
    return aa / t, (a / aa) * np.conj(b) / t


def fgmres(apply_A: Callable[[np.ndarray], np.ndarray], apply_M: Callable[[np.ndarray], np.ndarray],
           b: np.ndarray, restart: int, rtol: float, max_iters: int,
           x0: Optional[np.ndarray] = None, reorth: str = "always") -> FGMRESResult:
    """Restarted right-preconditioned flexible GMRES with CGS2 (Sec. 3 outer solver).

    Each Arnoldi step: z_j = M v_j, w = A z_j, h = V^H w, w -= V h,
    h' = V^H w, w -= V h', h += h', v_{j+1} = w / ||w||; the Givens rotations
    update g and the cycle stops at |g_{j+1}| <= rtol ||b||.  Then
    x += Z y with H y = g, and the true residual decides whether to restart.
    ``iters`` counts Arnoldi steps over all cycles.

    ``reorth="selective"`` runs the second Gram-Schmidt pass only when the first
    one left less than a tenth of ||w|| (Rutishauser's criterion); otherwise h' = 0.
    """
    if reorth not in ("always", "selective"):
        raise ValueError(reorth)
    b = np.asarray(b, dtype=np.complex128).ravel()
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).ravel().copy()
    if bnorm == 0.0:
        return FGMRESResult(x, 0, 0, True, 0.0, 0.0)
    iters, cycles, history = 0, 0, []
    relres_est = relres_true = 1.0
    while True:
        r = b - apply_A(x) if (x0 is not None or cycles > 0) else b.copy()
        beta = float(np.linalg.norm(r))
        relres_true = beta / bnorm
        if relres_true <= rtol or iters >= max_iters:
            return FGMRESResult(x, iters, cycles, relres_true <= rtol, relres_est, relres_true, history)
        V = np.zeros((restart + 1, b.size), dtype=np.complex128)
        Z = np.zeros((restart, b.size), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(restart):
            Z[j] = apply_M(V[j]).ravel()
            w = apply_A(Z[j])
            w_norm = float(np.linalg.norm(w))
            h = V[:j + 1].conj() @ w
            w = w - V[:j + 1].T @ h
            if reorth == "always" or np.linalg.norm(w) < 0.1 * w_norm:
                h2 = V[:j + 1].conj() @ w
                w = w - V[:j + 1].T @ h2
                h = h + h2
            hn = float(np.linalg.norm(w))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):
                t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t0
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            relres_est = abs(g[j + 1]) / bnorm
            history.append(relres_est)
            if relres_est <= rtol or hn == 0.0 or iters >= max_iters:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):                      # back substitution H y = g
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        cycles += 1


@dataclass
class BlockFGMRESResult:
    x: np.ndarray                 # [p, n]
    iters: int                    # block Arnoldi steps over all cycles
    restarts: int
    converged: np.ndarray         # [p] bool
    relres_est: np.ndarray        # [p]
    relres_true: np.ndarray       # [p]
    history: List[np.ndarray] = field(default_factory=list)


def block_fgmres(apply_A: Callable[[np.ndarray], np.ndarray], apply_M: Callable[[np.ndarray], np.ndarray],
                 B: np.ndarray, restart: int, rtol: float, max_iters: int) -> BlockFGMRESResult:
    """Restarted right-preconditioned block flexible GMRES for A X = B with p
    right-hand sides sharing one Krylov space (the outer solver of Sec. 3 taken to many
    sources at once; the block method itself is the textbook one, e.g. Saad, *Iterative
    Methods for Sparse Linear Systems*, 2nd ed., Sec. 6.12, made flexible as in Sec. 9.4).

    Per cycle: R = B - A X and R = V_0 S (thin QR, V_0 n x p); block Arnoldi step j:
    Z_j = M V_j (M applied to every column), W = A Z_j, H_ij = V_i^H W for all i <= j from the
    same W, then W -= sum_i V_i H_ij, the whole pass twice (block classical Gram-Schmidt, as
    the point FGMRES), W = V_{j+1} H_{j+1,j} (thin QR); Y
    minimises || E_1 S - Hbar_j Y ||_F (least squares) and the column norms of that
    residual are the columns' residual estimates.  The cycle ends when every column's
    estimate is <= rtol ||b_c|| (or at the restart, or when a new block is rank
    deficient); then X += [Z_0 .. Z_j] Y and the true residual decides whether to restart.
    x0 = 0.  ``iters`` counts block Arnoldi steps.
    """
    B = np.asarray(B, dtype=np.complex128)
    p = B.shape[0]
    Bm = B.reshape(p, -1).T                                  # n x p, columns are right-hand sides
    n = Bm.shape[0]
    bnorm = np.linalg.norm(Bm, axis=0)
    X = np.zeros_like(Bm)
    iters, cycles, history = 0, 0, []
    est = np.ones(p)
    A_cols = lambda M_: np.stack([apply_A(M_[:, c]) for c in range(M_.shape[1])], axis=1)
    M_cols = lambda M_: np.stack([np.asarray(apply_M(M_[:, c])).ravel() for c in range(M_.shape[1])], axis=1)
    while True:
        R = Bm - A_cols(X) if cycles > 0 else Bm.copy()
        true = np.linalg.norm(R, axis=0) / np.where(bnorm > 0, bnorm, 1.0)
        if np.all(true <= rtol) or iters >= max_iters:
            return BlockFGMRESResult(X.T.reshape(B.shape), iters, cycles, true <= rtol, est, true, history)
        V0, S = np.linalg.qr(R)
        V, Z = [V0], []
        Hbar = np.zeros(((restart + 1) * p, restart * p), dtype=np.complex128)
        E1S = np.zeros(((restart + 1) * p, p), dtype=np.complex128)
        E1S[:p] = S
        k = 0
        Y = np.zeros((0, p), dtype=np.complex128)
        for j in range(restart):
            Z.append(M_cols(V[j]))
            W = A_cols(Z[j])
            wnorm = np.linalg.norm(W)
            for _ in range(2):                               # classical: every H_ij from the same W
                Hs = [V[i].conj().T @ W for i in range(j + 1)]
                for i in range(j + 1):
                    W = W - V[i] @ Hs[i]
                    Hbar[i * p:(i + 1) * p, j * p:(j + 1) * p] += Hs[i]
            Vn, Hn = np.linalg.qr(W)
            Hbar[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Hn
            V.append(Vn)
            iters += 1
            k = j + 1
            rows, cols = (k + 1) * p, k * p
            Y = np.linalg.lstsq(Hbar[:rows, :cols], E1S[:rows], rcond=None)[0]
            est = np.linalg.norm(E1S[:rows] - Hbar[:rows, :cols] @ Y, axis=0) / np.where(bnorm > 0, bnorm, 1.0)
            history.append(est.copy())
            # a direction of the new block that Gram-Schmidt cancelled to rounding level: the
            # block Krylov space stops growing there (no deflation: the cycle ends)
            deficient = np.min(np.abs(np.diag(Hn))) <= 1e-12 * max(wnorm, 1e-300)
            if np.all(est <= rtol) or deficient or iters >= max_iters:
                break
        X = X + np.concatenate(Z[:k], axis=1) @ Y
        cycles += 1
