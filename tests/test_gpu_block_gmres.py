"""Block flexible GMRES on the GPU (hd_block_gmres_solve, through the C ABI) against the
oracle's block_fgmres (one Krylov space for several sources, block classical
Gram-Schmidt twice) and against the point FGMRES.

Tolerances as for the point solver: with FP64 factors the iterate after a fixed number of
block steps agrees to 1e-9 (the same block Krylov space and least-squares minimiser; the
bases differ by the thin QR's column phases, which the iterate does not see); with
complex FP32 factors the converged solutions agree with the FP64 oracle to 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import DDMPreconditioner, Grid, block_fgmres, fgmres, global_operator, rhs_from_source
from tests._cases import CASES, cuts, omega, velocity

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_02897_gb300.build import build  # noqa: E402

build()
from paper_1508_02897_gb300 import _binding as B  # noqa: E402
from paper_1508_02897_gb300.solver import HelmholtzDDM  # noqa: E402


def rel(a, b):
    a = np.asarray(a).ravel(); b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


_oracles = {}


def oracle(name):
    if name not in _oracles:
        case = CASES[name]
        c = velocity(case)
        g = Grid(case["N"], case["npml"], omega(case, c))
        A = global_operator(g, c)
        P = DDMPreconditioner(g, c, cuts(case), cuts(case), case["overlap"])
        _oracles[name] = (case, c, g, A, P)
    return _oracles[name]


def gpu(name, precision):
    case, c, g, _, _ = oracle(name)
    return HelmholtzDDM(case["N"], case["npml"], g.omega, c, case["nb"], case["nb"], case["overlap"],
                        precision=precision, cut_x=cuts(case), cut_y=cuts(case))


def sources(case, g, p, seed):
    rng = np.random.default_rng(seed)
    N, npml = case["N"], case["npml"]
    return np.stack([rhs_from_source(g, W.gaussian_source(N, npml, *rng.uniform(0.2, 0.8, 2), 2.0 / N))
                     for _ in range(p)])


@pytest.mark.parametrize("name", ["layers4", "ragged"])
def test_block_iterate_after_fixed_steps_c128(name):
    """Three sources, restart 3, four block steps (one restart inside): the GPU iterate is
    the oracle's."""
    case, c, g, A, P = oracle(name)
    Bm = sources(case, g, 3, seed=11)
    ref = block_fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), Bm, restart=3, rtol=1e-15, max_iters=4)
    s = gpu(name, "c128")
    x, st = s.block_solve(torch.from_numpy(Bm), restart=3, rtol=1e-15, max_iters=4)
    assert ref.iters == 4 and all(t["iters"] == 4 for t in st)
    assert rel(x.cpu().numpy(), ref.x.reshape(Bm.shape)) < 1e-9


def test_block_converged_c128_matches_oracle():
    case, c, g, A, P = oracle("layers4")
    Bm = sources(case, g, 3, seed=12)
    ref = block_fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), Bm, restart=10, rtol=1e-8, max_iters=200)
    s = gpu("layers4", "c128")
    x, st = s.block_solve(torch.from_numpy(Bm), restart=10, rtol=1e-8, max_iters=200)
    xn = x.cpu().numpy()
    assert all(t["converged"] == 1 for t in st)
    assert abs(st[0]["iters"] - ref.iters) <= 1
    for k in range(3):
        assert np.linalg.norm(Bm[k].ravel() - A @ xn[k].ravel()) / np.linalg.norm(Bm[k]) <= 1e-8


@pytest.mark.parametrize("precision", ["c64s", "c64"])
def test_block_mixed_precision_matches_fp64_oracle(precision):
    """Complex FP32 factors, FP64 block Gram-Schmidt and least squares: FP64 residual to 1e-8
    and solutions within 1e-5 of the oracle's FP64 FGMRES per source."""
    case, c, g, A, P = oracle("layers4")
    Bm = sources(case, g, 4, seed=13)
    sy = precision.endswith("s")
    s = HelmholtzDDM(case["N"], case["npml"], g.omega, c, case["nb"], case["nb"], case["overlap"],
                     precision="c64", cut_x=cuts(case), cut_y=cuts(case), symmetric=sy)
    x, st = s.block_solve(torch.from_numpy(Bm), restart=10, rtol=1e-8, max_iters=300)
    xn = x.cpu().numpy()
    for k in range(4):
        assert st[k]["converged"] == 1
        assert np.linalg.norm(Bm[k].ravel() - A @ xn[k].ravel()) / np.linalg.norm(Bm[k]) <= 1e-8
        ref = fgmres(lambda v: A @ v, lambda v: P.apply(v).ravel(), Bm[k], restart=50, rtol=1e-10, max_iters=400)
        assert rel(xn[k], ref.x) < 1e-5


def test_block_of_one_is_point_fgmres():
    """p = 1: the block method is FGMRES with CGS2; after a fixed number of steps its iterate
    is the point solver's (FP64 Gram-Schmidt, both passes)."""
    case, c, g, A, P = oracle("ragged")
    b = sources(case, g, 1, seed=14)
    s = gpu("ragged", "c128")
    xb, stb = s.block_solve(torch.from_numpy(b), restart=4, rtol=1e-15, max_iters=6)
    xp, stp = s.solve(torch.from_numpy(b[0]), restart=4, rtol=1e-15, max_iters=6, arnoldi="fp64", reorth="always")
    assert stb[0]["iters"] == stp[0]["iters"] == 6
    assert rel(xb.cpu().numpy()[0], xp.cpu().numpy()) < 1e-9


def test_block_fewer_steps_than_point_iterations():
    """The block space holds every source's Krylov space: the block solve needs no more block
    steps than the largest per-source FGMRES iteration count."""
    case, c, g, A, P = oracle("layers4")
    Bm = sources(case, g, 4, seed=15)
    s = gpu("layers4", "c64")
    _, stb = s.block_solve(torch.from_numpy(Bm), restart=20, rtol=1e-8, max_iters=300)
    _, stp = s.solve(torch.from_numpy(Bm), restart=20, rtol=1e-8, max_iters=300)
    assert all(t["converged"] == 1 for t in stb + stp)
    assert stb[0]["iters"] <= max(t["iters"] for t in stp)
