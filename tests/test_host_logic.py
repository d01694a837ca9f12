"""Host-side logic that needs no GPU: the seeded workload generators and the
byte models the bench divides by (roofline numerators)."""
import numpy as np

import bench
import workloads as W


def test_workloads_are_seeded_and_shaped():
    a = W.make_workload("precision")
    b = W.make_workload("precision")
    assert a.n == 4096 + 32 and a.c.shape == (a.n, a.n) and a.f.shape == (1, a.n, a.n)
    assert np.array_equal(a.c, b.c) and np.array_equal(a.f, b.f)
    assert 0.7 - 1e-12 <= a.c.min() and a.c.max() <= 1.3 + 1e-12       # c = 1 + 0.3 clip(g, -1, 1)
    bt = W.make_workload("batching", nrhs=64)      # the bench asks for its 64 sources
    assert bt.N == 1984 and bt.nrhs == 64 and bt.nbx == bt.nby == 16
    peaks = {tuple(np.unravel_index(np.argmax(np.abs(f)), f.shape)) for f in bt.f}
    assert len(peaks) == 64                       # 64 distinct seeded source positions
    widths = np.diff(bt.cut_x)
    assert widths[0] == widths[-1] == 96 and np.all(widths[1:-1] == 128)   # uneven edge boxes
    md = W.make_workload("medium")
    assert set(np.unique(md.c)) <= {1.0, 1.5, 2.0}                        # three layers


def test_box_extents_match_the_decomposition():
    """Interior boxes: owned 128 + 2 (overlap 8 + PML 16) = 176; boxes at the edge of
    the grid: 128 + 16 (global PML owned) + 8 + 16 = 168."""
    wl = W.make_workload("precision")
    ext = [bench._extent(wl.cut_x, i, wl) for i in range(wl.nbx)]
    assert ext[0] == ext[-1] == 168 and all(e == 176 for e in ext[1:-1])


def test_block_entries_per_storage():
    assert bench.block_entries(176, "full") == 176 * 176
    assert bench.block_entries(176, False) == 176 * 176
    assert bench.block_entries(176, "sym") == 11 * 12 // 2 * 256          # upper 16x16 tiles
    assert bench.block_entries(168, "sym") == 11 * 12 // 2 * 256
    assert bench.block_entries(170, "tc") == 176 * 176                    # rounded up to 8
    assert bench.block_entries(176, "sym") < 0.55 * 176 * 176


def test_subst_bytes_counts_each_block_forward_and_backward():
    """One box, one source: (2 rows - 1) blocks of the stored entries, the owned residual
    read once (16 B per cell of the grid) and the staging vector written, read and
    rewritten (3 rows m c)."""
    wl = W.make_workload("tiny", N=64, nb=1)
    m = rows = bench._extent(wl.cut_x, 0, wl)
    assert m == 64 + 32
    got = bench.subst_bytes(wl, 8, 1, 8, "full")
    assert got == 16 * wl.n * wl.n + (2 * rows - 1) * m * m * 8 + 3 * rows * m * 8
    # 16 sources: groups of 8 per CTA on the CUDA cores (factor read twice), 16 on the tensor cores (once)
    g16 = bench.subst_bytes(wl, 8, 16, 8, "full") - 16 * (16 * wl.n * wl.n + 3 * rows * m * 8)
    t16 = bench.subst_bytes(wl, 8, 16, 8, "tc") - 16 * (16 * wl.n * wl.n + 3 * rows * m * 8)
    assert g16 == 2 * (2 * rows - 1) * m * m * 8 and t16 == (2 * rows - 1) * m * m * 8
    # 64 sources: 8 groups on the CUDA cores, 4 of 16 on the tensor cores
    t64 = bench.subst_bytes(wl, 8, 64, 8, "tc") - 64 * (16 * wl.n * wl.n + 3 * rows * m * 8)
    assert t64 == 4 * (2 * rows - 1) * m * m * 8


def test_arnoldi_step_indices_follow_the_cycles():
    assert bench._arnoldi_js(0, 10) == []
    assert bench._arnoldi_js(3, 10) == [0, 1, 2]
    assert bench._arnoldi_js(23, 10) == list(range(10)) * 2 + [0, 1, 2]


def test_solve_starts_from_x0_when_out_is_given(monkeypatch):
    """HelmholtzDDM.solve hands the C ABI the initial guess in the output buffer: with
    both out and x0 the buffer must hold x0 (host logic only: the ABI call is stubbed)."""
    import torch
    from paper_1508_02897_gb300 import solver as S
    seen = {}

    def fake_solve(ctx, b_ptr, x_ptr, nrhs, *args, **kw):
        seen["use_x0"] = kw["use_x0"]
        return 0, []

    monkeypatch.setattr(S.B, "hd_gmres_solve", fake_solve)
    monkeypatch.setattr(S, "_stream_ptr", lambda stream: 0)
    s = S.HelmholtzDDM.__new__(S.HelmholtzDDM)
    s.n, s.device, s.stream, s.prec, s.ctx = 4, torch.device("cpu"), None, S.B.HD_C64, None
    s.scratch, s.scratch_bytes = torch.empty(16, dtype=torch.uint8), 16
    s._krylov = {(5, 1): torch.empty(16, dtype=torch.uint8)}
    b = torch.ones((4, 4), dtype=torch.complex128)
    x0 = torch.full((4, 4), 2 + 1j, dtype=torch.complex128)
    out = torch.zeros((4, 4), dtype=torch.complex128)
    x, _ = s.solve(b, restart=5, x0=x0, out=out)
    assert x is out and torch.equal(out, x0) and seen["use_x0"] == 1
    x, _ = s.solve(b, restart=5, out=torch.zeros((4, 4), dtype=torch.complex128))
    assert seen["use_x0"] == 0



def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host cores) prints one JSON
    line with the contract's keys, its own cpu_baseline and an e2e object without
    host-device traffic."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("precision")
