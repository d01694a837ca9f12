"""Tensor-core factorisation of the Schur blocks (pivot-free blocked Gauss-Jordan with
tcgen05 MMAs, hd_factor_tc.cu) through the C ABI: preconditioner applications built on
its factors against the FP64 oracle and against the SIMT kernel with partial pivoting,
in every storage of complex FP32 arithmetic, plus the pivot check's fallback.

Tolerances as in test_gpu_parity: complex FP32 factors 2e-4 relative L2 per
application (FP32 rounding times the local condition number; the BF16x3 split products
are FP32-grade, the tensor cores' FP32 accumulation truncates), FP16 and TF32 storage
3e-2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import DDMPreconditioner, Grid
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
        _oracles[name] = (case, c, g, DDMPreconditioner(g, c, cuts(case), cuts(case), case["overlap"]))
    return _oracles[name]


def gpu(name, precision, path, pivot_ratio=0.5):
    case, c, g, _ = oracle(name)
    return HelmholtzDDM(case["N"], case["npml"], g.omega, c, case["nb"], case["nb"], case["overlap"],
                        precision=precision.rstrip("st"), cut_x=cuts(case), cut_y=cuts(case),
                        symmetric=precision.endswith("s"), tcore=precision.endswith("t"),
                        factor_path=path, pivot_ratio=pivot_ratio)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["c64", "c64s", "c64h", "c64hs", "c64t"])
def test_tcore_factor_matches_oracle_and_simt(name, precision):
    case, _, g, P = oracle(name)
    nsub = case["nb"] ** 2
    r = W.random_complex((g.n, g.n), seed=41)
    ref = P.apply(r)
    s_tc = gpu(name, precision, "tcore")
    assert s_tc.factor_report() == (nsub, 0), "no pivot of these Schur blocks should fail the check"
    z_tc = s_tc.apply_precond(torch.from_numpy(r)).cpu().numpy()
    s_si = gpu(name, precision, "simt")
    assert s_si.factor_report() == (0, nsub)
    z_si = s_si.apply_precond(torch.from_numpy(r)).cpu().numpy()
    e_tc, e_si = rel(z_tc, ref), rel(z_si, ref)
    tol = 2e-4 if precision in ("c64", "c64s") else 3e-2
    assert e_tc < tol and e_si < tol, (e_tc, e_si)
    if precision in ("c64", "c64s"):
        # FP32-grade: the BF16x3 products are exact to 2^-25, but the tensor cores truncate
        # (round toward zero) each FP32 accumulation, and an entry of the trailing matrix
        # passes through 24 MMAs per 16-column panel: within ten times the error of the
        # FP32 Gauss-Jordan on the CUDA cores (measured: about 4x)
        assert e_tc < 10 * e_si + 1e-7, (e_tc, e_si)


def test_auto_path_uses_tensor_cores_for_complex_fp32():
    case, _, g, _ = oracle("wide")
    s = gpu("wide", "c64s", "auto")
    assert s.factor_report() == (case["nb"] ** 2, 0)
    s128 = gpu("wide", "c128", "auto")
    assert s128.factor_report() == (0, case["nb"] ** 2)


def test_tcore_path_refused_for_fp64_factors():
    with pytest.raises(B.HDError) as e:
        gpu("tiny", "c128", "tcore")
    assert e.value.code == B.HD_ERR_INVALID


@pytest.mark.parametrize("precision", ["c64s", "c64t"])
def test_pivot_check_refactors_marked_boxes(precision):
    """A pivot ratio no pivot can meet marks every box: the same call then refactorises
    all of them with partial pivoting, so the result is bitwise the SIMT kernel's."""
    case, _, g, P = oracle("wide")
    nsub = case["nb"] ** 2
    r = W.random_complex((g.n, g.n), seed=43)
    s_all = gpu("wide", precision, "auto", pivot_ratio=1e30)
    assert s_all.factor_report() == (0, nsub)
    s_si = gpu("wide", precision, "simt")
    z_all = s_all.apply_precond(torch.from_numpy(r)).cpu().numpy()
    z_si = s_si.apply_precond(torch.from_numpy(r)).cpu().numpy()
    assert np.array_equal(z_all, z_si)


def test_tcore_factor_is_deterministic():
    """Two factorisations of the same medium give bitwise the same factors."""
    _, _, g, _ = oracle("wide")
    r = W.random_complex((g.n, g.n), seed=47)
    z = [gpu("wide", "c64s", "tcore").apply_precond(torch.from_numpy(r)).cpu().numpy() for _ in range(2)]
    assert np.array_equal(z[0], z[1])
