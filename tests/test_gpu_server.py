"""Serving loop (hd_server_*): concurrent requests of different grids, media
and source counts; each result equals the same request solved alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import workloads as W  # noqa: E402
from oracle import Grid, global_operator, rhs_from_source  # noqa: E402
from paper_1508_02897_gb300.build import build  # noqa: E402

build()
from paper_1508_02897_gb300.solver import Server  # noqa: E402


def _request(N, medium, nrhs, seed):
    wl = W.make_workload("tiny", N=N, nb=N // 64, medium=medium, seed=seed, nrhs=nrhs)
    return wl


def test_alone_equals_in_the_mix():
    reqs = [_request(128, "homogeneous", 1, 0), _request(192, "three_layer", 3, 1), _request(256, "random", 2, 2),
            _request(128, "random", 4, 3)]
    srv = Server(hbm_budget_bytes=8 << 30, max_slots=4)
    alone = []
    for wl in reqs:   # one at a time
        t = srv.submit(wl.c, wl.f, wl.N, wl.npml, wl.omega, wl.nbx, wl.nby, wl.overlap, 30, 1e-8)
        alone.append(srv.poll(t))
    tickets = [srv.submit(wl.c, wl.f, wl.N, wl.npml, wl.omega, wl.nbx, wl.nby, wl.overlap, 30, 1e-8) for wl in reqs]
    mixed = [srv.poll(t) for t in tickets]
    info = srv.info()
    srv.close()
    assert info["completed"] == 2 * len(reqs) and info["peak_running"] >= 2
    for wl, (xa, sa, _), (xm, sm, im) in zip(reqs, alone, mixed):
        assert np.array_equal(xa, xm)
        assert [s["iters"] for s in sa] == [s["iters"] for s in sm]
        g = Grid(wl.N, wl.npml, wl.omega)
        A = global_operator(g, wl.c)
        for k in range(wl.nrhs):
            b = rhs_from_source(g, wl.f[k]).ravel()
            assert sm[k]["converged"] == 1
            assert np.linalg.norm(b - A @ xm[k].ravel()) / np.linalg.norm(b) <= 1e-8
        assert im["latency_s"] >= im["run_s"] > 0


def test_budget_splits_sources_and_rejects_oversize():
    wl = _request(256, "random", 4, 7)
    one = Server(hbm_budget_bytes=8 << 30, max_slots=1)
    t = one.submit(wl.c, wl.f, wl.N, wl.npml, wl.omega, wl.nbx, wl.nby, wl.overlap, 30, 1e-8)
    x_all, s_all, i_all = one.poll(t)
    one.close()
    small = Server(hbm_budget_bytes=int(0.3e9), max_slots=2)   # room for about one source at a time
    t = small.submit(wl.c, wl.f, wl.N, wl.npml, wl.omega, wl.nbx, wl.nby, wl.overlap, 30, 1e-8)
    x_b, s_b, i_b = small.poll(t)
    assert i_b["batch"] < 4 and i_all["batch"] == 4
    assert np.array_equal(x_all, x_b)
    from paper_1508_02897_gb300 import _binding as B
    with pytest.raises(B.HDError) as e:
        big = W.make_workload("tiny", N=1024, nb=8)
        small.submit(big.c, big.f, big.N, big.npml, big.omega, big.nbx, big.nby, big.overlap, 30, 1e-8)
    assert e.value.code == B.HD_ERR_OOM
    small.close()
