"""The multi-GPU mode of the benchmark is replicas: every rank solves its own
source on the same medium, with no data-path collective; only the timing uses
a barrier and max/sum over ranks.  That host logic runs here as two gloo ranks
on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = type("A", (), dict(config="tiny", restart=None, rtol=None, nrhs=None))()
    wl = bench.workload(args, rank)
    mx = bench.max_over_ranks(float(rank + 1), world)
    sm = bench.sum_over_ranks(float(rank + 1), world)
    bench.barrier(world)
    out[rank] = (mx, sm, int(np.argmax(np.abs(wl.f))), float(wl.c.sum()), wl.f.shape)
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0            # max over ranks
    assert res[0][1] == res[1][1] == 3.0            # sum over ranks
    assert res[0][3] == res[1][3]                   # same medium on every rank
    assert res[0][2] != res[1][2]                   # each rank its own source position
    assert res[0][4] == res[1][4]
