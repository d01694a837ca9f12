"""Parity at the benchmark sizes, in the launch configuration the bench times.

The oracle cannot factorise all 1024 boxes of the 4096^2 workload in a test, so
these tests sample: a preconditioner output cell that lies in the owned part of
box b and outside every other box's extent is exactly box b's local solution
(Eq. (ddm0) and (pc)), which the oracle computes with one sparse LU of that box
alone.  Corner, edge and interior boxes are sampled.  The full solve is checked
through a property that holds at any size: its FP64 relative residual, formed on
the CPU with the oracle's own operator.

Tolerances as in test_gpu_parity: FP32 factors and the split-TF32 tensor-core
storage 2e-4 relative L2 per sampled box, TF32 tensor-core storage 3e-2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import DDMPreconditioner, Grid, global_operator, rhs_from_source

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_02897_gb300.build import build  # noqa: E402

build()
from paper_1508_02897_gb300 import _binding as B  # noqa: E402
from paper_1508_02897_gb300.solver import HelmholtzDDM  # noqa: E402


def _exclusive_cells(subs, b):
    """Owned cells of box b outside the extent of every other box."""
    s = subs[b]
    mask = np.zeros((s.oy1 - s.oy0, s.ox1 - s.ox0), bool)
    mask[:] = True
    for t, o in enumerate(subs):
        if t == b:
            continue
        y0, y1 = max(o.ey0, s.oy0), min(o.ey1, s.oy1)
        x0, x1 = max(o.ex0, s.ox0), min(o.ex1, s.ox1)
        if y0 < y1 and x0 < x1:
            mask[y0 - s.oy0:y1 - s.oy0, x0 - s.ox0:x1 - s.ox0] = False
    return mask


def _sampled_boxes(wl):
    nbx, nby = wl.nbx, wl.nby
    return [0, nbx - 1 + (nby // 2) * nbx, (nby // 2) * nbx + nbx // 2, nbx * nby - 1]   # corner, edge, interior, corner


def _check_boxes(wl, z, f, tol):
    g = Grid(wl.N, wl.npml, wl.omega)
    for b in _sampled_boxes(wl):
        P = DDMPreconditioner(g, wl.c, wl.cut_x, wl.cut_y, wl.overlap, subdomains=[b])
        s = P.subs[b]
        mask = _exclusive_cells(P.subs, b)
        assert mask.sum() > 1000
        u = P.local_solve(b, f)
        ref = u[s.oy0 - s.ey0:s.oy1 - s.ey0, s.ox0 - s.ex0:s.ox1 - s.ex0][mask]
        got = z[s.oy0:s.oy1, s.ox0:s.ox1][mask]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, (b, np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_precond_4096_sampled_boxes():
    """4096^2, 32x32 boxes, c64 factors in symmetric tile storage (the headline
    configuration): sampled boxes of one preconditioner application."""
    wl = W.make_workload("precision")
    s = HelmholtzDDM(wl.N, wl.npml, wl.omega, wl.c, wl.nbx, wl.nby, wl.overlap, precision="c64", cut_x=wl.cut_x,
                     cut_y=wl.cut_y, symmetric=True)
    f = W.random_complex((wl.n, wl.n), seed=41)
    z = s.apply_precond(torch.from_numpy(f)).cpu().numpy()
    s.close()
    _check_boxes(wl, z, f, 2e-4)


@pytest.mark.parametrize("tcore,nrhs,checked,tol", [(True, 16, (0, 15), 3e-2), ("x3", 40, (0, 31, 32, 39), 2e-4)])
def test_precond_batching_tensor_cores_sampled_boxes(tcore, nrhs, checked, tol):
    """1984^2, 16x16 uneven boxes, tensor-core storage, several sources in one
    application (the batching configuration's lockstep group): sampled boxes of some of
    the sources.  TF32 storage: 16 sources, one CTA group; split-TF32 (FP32-grade): 40
    sources, a full group of 32 and a ragged one of 8."""
    wl = W.make_workload("batching", nrhs=nrhs)
    s = HelmholtzDDM(wl.N, wl.npml, wl.omega, wl.c, wl.nbx, wl.nby, wl.overlap, precision="c64", cut_x=wl.cut_x,
                     cut_y=wl.cut_y, tcore=tcore)
    f = W.random_complex((nrhs, wl.n, wl.n), seed=43)
    _, _, need = B.hd_query_workspace(s.ctx, nrhs, 1)
    s.scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    s.scratch_bytes = need
    z = s.apply_precond(torch.from_numpy(f)).cpu().numpy()
    s.close()
    for k in checked:
        _check_boxes(wl, z[k], f[k], tol)


def test_solve_4096_residual_from_oracle_operator():
    """The headline solve (4096^2, c64 symmetric storage, double-single FGMRES(10),
    selective reorthogonalisation, rtol 1e-6): the relative residual of the GPU
    solution, formed in FP64 on the CPU with the oracle's operator, meets the
    tolerance, and the solver's own FP64 residual agrees with it."""
    wl = W.make_workload("precision")
    g = Grid(wl.N, wl.npml, wl.omega)
    s = HelmholtzDDM(wl.N, wl.npml, wl.omega, wl.c, wl.nbx, wl.nby, wl.overlap, precision="c64", cut_x=wl.cut_x,
                     cut_y=wl.cut_y, symmetric=True)
    b = rhs_from_source(g, wl.f[0])
    x, st = s.solve(torch.from_numpy(b), restart=wl.restart, rtol=wl.rtol, max_iters=1000)
    s.close()
    assert st[0]["converged"] == 1
    A = global_operator(g, wl.c)
    r = b.ravel() - A @ x.cpu().numpy().ravel()
    relres = np.linalg.norm(r) / np.linalg.norm(b)
    assert relres <= wl.rtol
    assert abs(relres - st[0]["relres_true"]) <= 1e-3 * relres
