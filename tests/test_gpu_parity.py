"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances: the c128 path follows the same arithmetic in FP64 with a different
direct solver (block Schur inverses vs. sparse LU), so results agree to
rounding times the local condition number: matvec 1e-13, preconditioner 1e-10
relative L2, FGMRES iterate after a fixed number of steps 1e-9.  The c64 path
stores the local factors in complex FP32: preconditioner 2e-4 relative L2
(FP32 rounding amplified by the local problems' condition number), final
solution 1e-5 against the FP64 oracle at relative residual 1e-8.  Reduced-precision
storage of the factors scales that bound by its unit roundoff over FP32's: TF32 and
FP16 storage (2^-11) 3e-2, BF16 storage (2^-8, eight times coarser) 1.2e-1; the FP64
outer loop still reaches its tolerance.  The split-TF32 tensor-core storage (c64x: hi/lo
TF32 pairs, products to about FP32's unit roundoff) keeps the FP32 bound, 2e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import DDMPreconditioner, Grid, fgmres, global_operator, rhs_from_source
from tests._cases import CASES, cuts, omega, velocity

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_02897_gb300.build import build  # noqa: E402

build()
from paper_1508_02897_gb300.solver import HelmholtzDDM  # noqa: E402


def rel(a, b):
    a = np.asarray(a).ravel(); b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


_oracles = {}


def oracle(name, own=True):
    key = (name, own)
    if key not in _oracles:
        case = CASES[name]
        c = velocity(case)
        g = Grid(case["N"], case["npml"], omega(case, c))
        A = global_operator(g, c)
        P = DDMPreconditioner(g, c, cuts(case), cuts(case), case["overlap"], own_global_pml=own)
        _oracles[key] = (case, c, g, A, P)
    return _oracles[key]


def gpu(name, precision, own=True):
    """precision: c128 / c64 / c64h, with a trailing "s" for symmetric tile storage,
    "t" for the tensor-core storage (c64t: TF32 factors, tcgen05 substitution) or "x"
    for the split-TF32 tensor-core storage (c64x: FP32-grade products)."""
    case, c, g, _, _ = oracle(name, own)
    sym = precision.endswith("s")
    tc = "x3" if precision.endswith("x") else precision.endswith("t")
    return HelmholtzDDM(case["N"], case["npml"], g.omega, c, case["nb"], case["nb"], case["overlap"],
                        precision=precision.rstrip("stx"), cut_x=cuts(case), cut_y=cuts(case), own_global_pml=own,
                        symmetric=sym, tcore=tc)


def _x3_fits(name):
    """The split-TF32 storage takes boxes up to 176 cells wide (the "wide" case has 178)."""
    return name != "wide"


@pytest.mark.parametrize("name", list(CASES))
def test_matvec_and_rhs(name):
    case, c, g, A, _ = oracle(name)
    s = gpu(name, "c128")
    x = W.random_complex((2, g.n, g.n), seed=7)
    y = s.matvec(torch.from_numpy(x)).cpu().numpy()
    for k in range(2):
        ref = (A @ x[k].ravel()).reshape(g.n, g.n)
        assert rel(y[k], ref) < 1e-13
    f = W.gaussian_source(case["N"], case["npml"], 0.3, 0.6, 2.0 / case["N"])
    b = s.rhs(torch.from_numpy(f)).cpu().numpy()
    assert rel(b, rhs_from_source(g, f)) < 1e-14


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64", 2e-4), ("c64h", 3e-2), ("c128s", 1e-10),
                                           ("c64s", 2e-4), ("c64hs", 3e-2), ("c64t", 3e-2), ("c64b", 1.2e-1),
                                           ("c64bs", 1.2e-1), ("c64x", 2e-4)])
def test_precond_parity(name, precision, tol):
    _, _, g, _, P = oracle(name)
    if precision == "c64x" and not _x3_fits(name):
        from paper_1508_02897_gb300._binding import HDError
        with pytest.raises(HDError):
            gpu(name, precision)
        return
    s = gpu(name, precision)
    r = W.random_complex((g.n, g.n), seed=3)
    z = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    ref = P.apply(r)
    assert rel(z, ref) < tol
    # deterministic: a second application is bitwise identical
    z2 = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    assert np.array_equal(z, z2)


def test_precond_literal_ownership():
    """Owned boxes on the interior only (the literal reading of Sec. 2)."""
    _, _, g, _, P = oracle("ragged", own=False)
    s = gpu("ragged", "c128", own=False)
    r = W.random_complex((g.n, g.n), seed=8)
    assert rel(s.apply_precond(torch.from_numpy(r)).cpu().numpy(), P.apply(r)) < 1e-10


@pytest.mark.parametrize("name", ["tiny", "ragged"])
@pytest.mark.parametrize("arnoldi", ["fp64", "ds"])
@pytest.mark.parametrize("reorth", ["always", "selective"])
@pytest.mark.parametrize("restart,k", [(3, 4), (10, 10)])
def test_gmres_fixed_steps_c128(name, arnoldi, reorth, restart, k):
    """Same FGMRES variant on both sides: the iterate after k steps agrees
    (FP64 Gram-Schmidt, and the double-single one whose basis carries ~48 bits;
    two passes always, or the second only after a cancellation).  A 10-step cycle
    runs the double-single dot kernel's 4-, 8- and 12-vector classes and the steps
    whose chunks hold more tiles than the ring has stages."""
    case, c, g, A, P = oracle(name)
    s = gpu(name, "c128")
    f = W.gaussian_source(case["N"], case["npml"], 0.45, 0.55, 2.0 / case["N"])
    b = rhs_from_source(g, f)
    ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, restart=restart, rtol=1e-15, max_iters=k,
                 reorth=reorth)
    x, st = s.solve(torch.from_numpy(b), restart=restart, rtol=1e-15, max_iters=k, arnoldi=arnoldi, reorth=reorth)
    assert st[0]["iters"] == ref.iters == k
    assert rel(x.cpu().numpy(), ref.x.reshape(g.n, g.n)) < 1e-9


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("arnoldi", ["fp64", "ds"])
@pytest.mark.parametrize("reorth", ["always", "selective"])
def test_gmres_converged_c128(name, arnoldi, reorth):
    case, c, g, A, P = oracle(name)
    s = gpu(name, "c128")
    f = W.gaussian_source(case["N"], case["npml"], 0.5, 0.5, 2.0 / case["N"])
    b = rhs_from_source(g, f)
    ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, restart=50, rtol=1e-8, max_iters=300, reorth=reorth)
    x, st = s.solve(torch.from_numpy(b), restart=50, rtol=1e-8, max_iters=300, arnoldi=arnoldi, reorth=reorth)
    assert st[0]["converged"] == 1 and abs(st[0]["iters"] - ref.iters) <= 1
    xn = x.cpu().numpy().ravel()
    assert np.linalg.norm(b.ravel() - A @ xn) / np.linalg.norm(b) <= 1e-8
    assert rel(xn, ref.x) < 1e-9


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["c64", "c64h", "c64s", "c64t", "c64bs", "c64x"])
def test_gmres_mixed_precision(name, precision):
    """FP32 local factors (stored in FP32, FP16, TF32 or split TF32), FP64 outer loop: the
    FP64 relative residual reaches the tolerance and the solution matches the FP64
    oracle to 1e-5."""
    case, c, g, A, P = oracle(name)
    if precision == "c64x" and not _x3_fits(name):
        pytest.skip("boxes wider than the split-TF32 storage takes")
    s = gpu(name, precision)
    f = W.gaussian_source(case["N"], case["npml"], 0.5, 0.5, 2.0 / case["N"])
    b = rhs_from_source(g, f)
    ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, restart=50, rtol=1e-10, max_iters=400)
    x, st = s.solve(torch.from_numpy(b), restart=50, rtol=1e-8, max_iters=400)
    xn = x.cpu().numpy().ravel()
    assert st[0]["converged"] == 1
    assert np.linalg.norm(b.ravel() - A @ xn) / np.linalg.norm(b) <= 1e-8
    assert rel(xn, ref.x) < 1e-5


def test_one_box_is_exact():
    """Nb = 1: the preconditioner is the exact PML solve, so one iteration."""
    N, npml = 96, 16
    c = W.velocity_random_field(N, npml, seed=4)
    om = 2 * np.pi * float(c.min()) * N / 10
    g = Grid(N, npml, om)
    A = global_operator(g, c)
    s = HelmholtzDDM(N, npml, om, c, 1, 1, 8, precision="c128")
    b = rhs_from_source(g, W.gaussian_source(N, npml, 0.4, 0.5, 2.0 / N))
    x, st = s.solve(torch.from_numpy(b), restart=10, rtol=1e-10, max_iters=20)
    assert st[0]["iters"] == 1 and st[0]["converged"] == 1
    xn = x.cpu().numpy().ravel()
    assert np.linalg.norm(b.ravel() - A @ xn) / np.linalg.norm(b) < 1e-11


# ---------------------------------------------------------------- several right-hand sides
def _sources(case, k, seed):
    rng = np.random.default_rng(seed)
    N, npml = case["N"], case["npml"]
    return np.stack([W.gaussian_source(N, npml, *rng.uniform(0.15, 0.85, 2), 2.0 / N) for _ in range(k)])


@pytest.mark.parametrize("precision,nrhs", [("c128", 3), ("c64", 9), ("c64s", 5), ("c64t", 5), ("c64t", 19),
                                             ("c64t", 37), ("c64x", 5), ("c64x", 70)])
def test_precond_batched_equals_single(precision, nrhs):
    """Each right-hand side of a batched application (groups of up to 8 per CTA, 16
    on the tensor cores; 37 sources there give two full groups and a ragged one of 5,
    launched side by side per box; 32 per CTA with the split-TF32 storage, 70 sources
    giving two full groups and a ragged one of 6) gives bitwise the same vector as its
    own application."""
    _, _, g, _, P = oracle("ragged")
    s = gpu("ragged", precision)
    r = W.random_complex((nrhs, g.n, g.n), seed=12)
    from paper_1508_02897_gb300 import _binding as B
    _, _, need = B.hd_query_workspace(s.ctx, nrhs, 1)
    s.scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    s.scratch_bytes = need
    z = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    for k in range(nrhs):
        zk = s.apply_precond(torch.from_numpy(r[k])).cpu().numpy()
        assert np.array_equal(z[k], zk)
    tol = 1e-10 if precision.startswith("c128") else (3e-2 if precision.endswith("t") else 2e-4)
    if precision == "c64x":   # every source in the groups of 32 against the oracle
        for k in (0, 31, 32, nrhs - 1) if nrhs > 32 else range(nrhs):
            assert rel(z[k], P.apply(r[k])) < tol
    assert rel(z[nrhs - 1], P.apply(r[nrhs - 1])) < tol


@pytest.mark.parametrize("precision", ["c128", "c64", "c64t", "c64x"])
def test_gmres_batched_alone_vs_mix(precision):
    """Lockstep solve of several sources sharing one factorisation: every
    solution is bitwise the one its source gets alone, and matches the oracle."""
    case, c, g, A, P = oracle("layers4")
    s = gpu("layers4", precision)
    f = _sources(case, 3, seed=5)
    b = np.stack([rhs_from_source(g, fk) for fk in f])
    xb, stb = s.solve(torch.from_numpy(b), restart=20, rtol=1e-8, max_iters=300)
    xb = xb.cpu().numpy()
    for k in range(3):
        xk, stk = s.solve(torch.from_numpy(b[k]), restart=20, rtol=1e-8, max_iters=300)
        assert stb[k]["iters"] == stk[0]["iters"] and stb[k]["converged"] == 1
        assert np.array_equal(xb[k], xk.cpu().numpy())
        assert np.linalg.norm(b[k].ravel() - A @ xb[k].ravel()) / np.linalg.norm(b[k]) <= 1e-8
    ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b[1], restart=20, rtol=1e-10, max_iters=400)
    assert rel(xb[1].ravel(), ref.x) < (1e-7 if precision == "c128" else 1e-5)


def test_autotune_keeps_results():
    """The autotuner only changes the launch shape: results stay bitwise identical."""
    _, _, g, _, P = oracle("layers4")
    s = gpu("layers4", "c64")
    r = W.random_complex((g.n, g.n), seed=31)
    z0 = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    threads, stages, ms = s.autotune()
    assert threads in (96, 128, 192, 256) and 2 <= stages <= 32
    z1 = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    assert np.array_equal(z0, z1)


@pytest.mark.parametrize("precision,reorth", [("c128", "always"), ("c64", "selective"), ("c128", "selective")])
def test_gmres_graph_capture_matches_launches(precision, reorth):
    """Arnoldi steps captured once as CUDA graphs and replayed (second solve on the
    same workspace) give bitwise the solution of plain launches."""
    case, c, g, A, P = oracle("ragged")
    s = gpu("ragged", precision)
    b = rhs_from_source(g, W.gaussian_source(case["N"], case["npml"], 0.35, 0.6, 2.0 / case["N"]))
    x0, st0 = s.solve(torch.from_numpy(b), restart=10, rtol=1e-9, max_iters=200, reorth=reorth)
    x1, st1 = s.solve(torch.from_numpy(b), restart=10, rtol=1e-9, max_iters=200, graphs=True, reorth=reorth)
    x2, st2 = s.solve(torch.from_numpy(b), restart=10, rtol=1e-9, max_iters=200, graphs=True, reorth=reorth)
    assert st0[0]["iters"] == st1[0]["iters"] == st2[0]["iters"] and st2[0]["converged"] == 1
    assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())
    assert np.array_equal(x0.cpu().numpy(), x2.cpu().numpy())


# ---------------------------------------------------------------- multi-step DDM
@pytest.mark.parametrize("name", ["ragged", "layers4"])
@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64s", 5e-4), ("c64t", 5e-2), ("c64x", 5e-4)])
def test_multistep_ddm_parity(name, precision, tol):
    """hd_apply_ddm (residual correction on the GPU) against the oracle's literal
    Eq. (ddms) (neighbour residuals per box) for 1, 2 and 3 steps, two sources."""
    _, _, g, _, P = oracle(name)
    s = gpu(name, precision)
    f = W.random_complex((2, g.n, g.n), seed=17)
    for steps in (1, 2, 3):
        u = s.apply_ddm(torch.from_numpy(f), steps).cpu().numpy()
        for k in range(2):
            assert rel(u[k], P.apply_multistep(f[k], steps)) < tol


def test_gmres_multistep_preconditioner():
    """FGMRES with the two-step DDM as preconditioner: the same iterate after k steps
    as the oracle's FGMRES with M = Eq. (ddms) + (sum) for two steps, and
    convergence in fewer iterations than the one-step preconditioner."""
    case, c, g, A, P = oracle("layers4")
    s = gpu("layers4", "c128")
    b = rhs_from_source(g, W.gaussian_source(case["N"], case["npml"], 0.4, 0.55, 2.0 / case["N"]))
    k = 4
    ref = fgmres(lambda v: A @ v, lambda v: P.apply_multistep(v, 2).ravel(), b, restart=3, rtol=1e-15, max_iters=k)
    x, st = s.solve(torch.from_numpy(b), restart=3, rtol=1e-15, max_iters=k, arnoldi="fp64", precond_steps=2)
    assert st[0]["iters"] == ref.iters == k
    assert rel(x.cpu().numpy(), ref.x.reshape(g.n, g.n)) < 1e-9
    _, st1 = s.solve(torch.from_numpy(b), restart=50, rtol=1e-8, max_iters=300)
    x2, st2 = s.solve(torch.from_numpy(b), restart=50, rtol=1e-8, max_iters=300, precond_steps=2)
    assert st2[0]["converged"] == 1 and st2[0]["iters"] < st1[0]["iters"]
    assert np.linalg.norm(b.ravel() - A @ x2.cpu().numpy().ravel()) / np.linalg.norm(b) <= 1e-8


# ---------------------------------------------------------------- smoothing function beta
def _gpu_smooth(name, precision):
    case, c, g, _, _ = oracle(name)
    return HelmholtzDDM(case["N"], case["npml"], g.omega, c, case["nb"], case["nb"], case["overlap"],
                        precision=precision.rstrip("st"), cut_x=cuts(case), cut_y=cuts(case),
                        symmetric=precision.endswith("s"), tcore=precision.endswith("t"), smoothing=True)


_smooth_oracles = {}


def _oracle_smooth(name):
    if name not in _smooth_oracles:
        case, c, g, A, _ = oracle(name)
        _smooth_oracles[name] = DDMPreconditioner(g, c, cuts(case), cuts(case), case["overlap"], smoothing=True)
    return _smooth_oracles[name]


@pytest.mark.parametrize("name", ["ragged", "layers4"])
@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64s", 2e-4), ("c64t", 3e-2)])
def test_precond_smoothing_parity(name, precision, tol):
    """HD_SMOOTH: every local solution weighted by beta_ij before the sum (Remark after
    Eq. (pc)), against the oracle's smoothed preconditioner; two sources."""
    _, _, g, _, _ = oracle(name)
    P = _oracle_smooth(name)
    s = _gpu_smooth(name, precision)
    r = W.random_complex((2, g.n, g.n), seed=19)
    z = s.apply_precond(torch.from_numpy(r)).cpu().numpy()
    for k in range(2):
        assert rel(z[k], P.apply(r[k])) < tol


def test_gmres_smoothing_fixed_steps_and_convergence():
    """FGMRES with the smoothed preconditioner: the iterate after k steps matches the
    oracle's FGMRES with the smoothed M (FP64 paths), and the solve converges."""
    case, c, g, A, _ = oracle("layers4")
    P = _oracle_smooth("layers4")
    s = _gpu_smooth("layers4", "c128")
    b = rhs_from_source(g, W.gaussian_source(case["N"], case["npml"], 0.45, 0.4, 2.0 / case["N"]))
    k = 4
    ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), b, restart=3, rtol=1e-15, max_iters=k)
    x, st = s.solve(torch.from_numpy(b), restart=3, rtol=1e-15, max_iters=k, arnoldi="fp64")
    assert st[0]["iters"] == ref.iters == k
    assert rel(x.cpu().numpy(), ref.x.reshape(g.n, g.n)) < 1e-9
    x2, st2 = s.solve(torch.from_numpy(b), restart=50, rtol=1e-8, max_iters=300)
    assert st2[0]["converged"] == 1
    assert np.linalg.norm(b.ravel() - A @ x2.cpu().numpy().ravel()) / np.linalg.norm(b) <= 1e-8
