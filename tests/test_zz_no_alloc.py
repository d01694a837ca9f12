"""The allocation-free preconditioner entry point, called through the C ABI.

Callers that cannot call cudaMalloc (plug-ins whose host application owns the
device heap, latency-bound loops where an allocation could synchronise the
device, services that must keep a fixed footprint after start-up) use
hd_apply_precond_noalloc, whose staging vectors live in a fixed 64 MiB array
inside the library.  Its result must match the
regular entry point, which stages through a caller workspace, bitwise, on two
calls in a row (the fixed array keeps the previous call's contents), in every
factor storage and when the sources do not fit the array at once.  This file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import workloads as W  # noqa: E402
from paper_1508_02897_gb300.build import build  # noqa: E402

build()
from paper_1508_02897_gb300 import _binding as B  # noqa: E402
from paper_1508_02897_gb300.solver import HelmholtzDDM  # noqa: E402


def _noalloc_fn():
    fn = B.lib().hd_apply_precond_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


# (precision, symmetric tiles, tensor-core storage, sources per call); the last case has more
# sources than the 64 MiB array holds at once (0.9 MB of staging each), so the entry point
# runs them in two groups
CASES = [("c128", False, False, 2), ("c64", False, False, 2), ("c64", True, False, 2), ("c64h", True, False, 2),
         ("c64h", False, False, 2), ("c64", False, True, 9), ("c64", False, "x3", 33), ("c64", True, False, 80)]


@pytest.mark.parametrize("precision,sym,tcore,nrhs", CASES)
def test_noalloc_matches_workspace_entry_point(precision, sym, tcore, nrhs):
    """Bitwise the result of hd_apply_precond with a caller workspace, on two calls in a
    row (the second must not see the first's leftovers in the shared array)."""
    N, npml, nb = 160, 16, 4
    c = W.velocity_random_field(N, npml, seed=21)
    omega = 2 * np.pi * float(c.min()) * N / 10
    s = HelmholtzDDM(N, npml, omega, c, nb, nb, 8, precision=precision, symmetric=sym, tcore=tcore)
    _, _, need = B.hd_query_workspace(s.ctx, nrhs, 1)
    s.scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    s.scratch_bytes = need
    st = int(torch.cuda.current_stream().cuda_stream)
    fn = _noalloc_fn()
    for seed in (1, 2):
        r = torch.from_numpy(W.random_complex((nrhs, s.n, s.n), seed=seed)).cuda()
        z_ref = s.apply_precond(r)
        z = torch.full_like(r, float("nan"))
        rc = fn(s.ctx, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), nrhs, ctypes.c_void_p(st))
        assert rc == B.HD_OK, B.hd_last_error()
        torch.cuda.synchronize()
        a, b = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)
    s.close()


def test_noalloc_rejects_oversize_problem():
    """A problem whose staging vectors exceed the fixed array is refused with HD_ERR_OOM."""
    N, npml, nb = 1536, 16, 12          # 144 boxes, 4.46M staging entries x 16 B > 64 MiB
    n = N + 2 * npml
    c = torch.ones((n, n), dtype=torch.float64, device="cuda")
    st = int(torch.cuda.current_stream().cuda_stream)
    ctx = B.hd_setup_medium(N, N, npml, 1.0 / N, 2 * np.pi * N / 10, c.data_ptr(), B.HD_C128, st, nb, nb, 8)
    fn = _noalloc_fn()
    r = torch.zeros((2, n, n), dtype=torch.complex128, device="cuda")
    rc = fn(ctx, ctypes.c_void_p(r[0].data_ptr()), ctypes.c_void_p(r[1].data_ptr()), 1, ctypes.c_void_p(st))
    assert rc == B.HD_ERR_OOM
    assert "64 MiB" in B.hd_last_error()
    B.hd_destroy(ctx)
