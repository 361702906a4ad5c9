"""The bench's multi-rank aggregation on CPU: two gloo ranks with different
timed durations; both see the slower one, and the value counts the work of
both ranks (weak scaling).  No GPU."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.aggregate(10.0 * (rank + 1), cells_per_rank=3e9, steps=2, world=world, device="cpu")
    dist.destroy_process_group()
    q.put((rank, out))


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, s, value = res[r]
        assert ms == 20.0                      # the slower rank's time
        assert abs(s - 0.01) < 1e-15           # 20 ms over 2 steps
        assert abs(value - 2 * 3e9 / 0.01 / 1e9) < 1e-9


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, s, value = bench.aggregate(50.0, cells_per_rank=1e9, steps=5, world=1)
    assert ms == 50.0 and abs(s - 0.01) < 1e-15 and abs(value - 100.0) < 1e-9


def test_roofline_entries_from_kernel_timings(monkeypatch):
    """bench.roofline: achieved = algorithmic bytes x cells / mean launch time,
    frac = achieved / measured peak, traffic (and its fraction) only for captured
    variants, the kernel with the larger share of the gradient first."""
    sys.path.insert(0, ROOT)
    import bench
    peak, kind = bench.peaks()
    info = {"padded_cells": 1_000_000, "ckpt_interval": 64, "stencil": 3, "adj_stencil": 1, "tile_x": 32,
            "tile_z": 16, "adj_tile_x": 32, "adj_tile_z": 16, "layout": 3, "staged_stores": 0, "adj_persistent": 1,
            "snap_store": 0, "stored_steps": 0}
    monkeypatch.setattr(bench, "TRAFFIC_PER_CELL", {("step", 3, 32, 16, 3, 0, 0): {"pass": 50.0, "keep": 60.0},
                                                    ("adj", 1, 32, 16, 1, 1, 0): 95.0})
    prof = {"step": (10.0, 100), "adj": (20.0, 50)}          # ms summed, launches timed
    first, second = bench.roofline("batched", info, prof, nt=4000, ns=32)
    step = first if first["kernel"].startswith("forward") else second
    adj = second if step is first else first
    assert abs(step["avg_us"] - 100.0) < 1e-9 and abs(adj["avg_us"] - 400.0) < 1e-9
    # sqrt(nt) checkpoints, FP32 velocities: half the forward launches keep v (60 and 68 B)
    assert step["bytes_per_cell"] == 64.0 and adj["bytes_per_cell"] == 108.0
    assert abs(step["achieved"] - 64.0 * 1e6 / 100e-6 / 1e9) < 1e-6
    assert abs(adj["achieved"] - 108.0 * 1e6 / 400e-6 / 1e9) < 1e-6
    assert abs(step["frac"] - step["achieved"] / peak) < 1e-12 and step["peak_kind"] == kind
    assert abs(step["frac_nominal"] - step["achieved"] / 7900.0) < 1e-12
    assert step["traffic"] == 55.0 * 1e6 and adj["traffic"] == 95.0 * 1e6
    assert abs(step["frac_traffic"] - 55.0 * 1e6 / 100e-6 / 1e9 / peak) < 1e-12
    # forward and recompute: 2 x 4000 x 100 us = 0.8 s against 4000 x 400 us = 1.6 s
    assert first is adj and abs(adj["time_share_est"] - 2 / 3) < 1e-12
    info2 = dict(info, layout=2)                             # a variant without a capture
    s2 = [r for r in bench.roofline("batched", info2, prof, nt=4000, ns=32) if r["kernel"].startswith("forward")][0]
    assert s2["traffic"] is None and s2["frac_traffic"] is None
    # the scaled-stress adjoint is another kernel: no traffic from the stress form's capture
    a2 = [r for r in bench.roofline("batched", dict(info, adj_form=2), prof, nt=4000, ns=32)
          if r["kernel"].startswith("adjoint")][0]
    assert a2["traffic"] is None and "scaled-stress" in a2["kernel"] and a2["bytes_per_cell"] == 108.0
    # every step stored with FP16 snapshots: 60 + 4 B forward, 100 + 4 B adjoint
    info3 = dict(info, ckpt_interval=4000, snap_store=1)
    r3 = {r["kernel"].split(" ")[0]: r for r in bench.roofline("batched", info3, prof, nt=4000, ns=32)}
    assert r3["forward_step"]["bytes_per_cell"] == 64.0 and r3["adjoint_step"]["bytes_per_cell"] == 104.0
    assert r3["forward_step"]["traffic"] is None             # captured with other snapshots
    # sqrt(nt) checkpoints with the final 3000 steps kept by the forward pass: 5000 forward
    # launches (4000 + 1000 recomputed), 4000 of which keep v: 60 + 8 x 4000 / 5000 B;
    # traffic mixes 1000 passes at 50 B with 4000 keeps at 60 B
    info4 = dict(info, stored_steps=3000)
    r4 = {r["kernel"].split(" ")[0]: r for r in bench.roofline("batched", info4, prof, nt=4000, ns=32)}
    assert abs(r4["forward_step"]["bytes_per_cell"] - 66.4) < 1e-12
    assert abs(r4["forward_step"]["traffic"] - (1000 * 50.0 + 4000 * 60.0) / 5000 * 1e6) < 1e-6
    assert abs(r4["adjoint_step"]["time_share_est"] - 1.6 / (1.6 + 0.5)) < 1e-12


def test_gradient_roofline_bytes_and_fractions():
    """bench.gradient_roofline: 236 B per padded cell-step with sqrt(nt) checkpoints
    (forward, recompute with the velocity hand-off, adjoint), 176 B with every step
    stored, 168 B with FP16 snapshots of every step; the floor fraction always uses
    176 B."""
    sys.path.insert(0, ROOT)
    import bench
    peak, _ = bench.peaks()
    info = {"padded_cells": 2_000_000, "ckpt_interval": 64, "stored_steps": 0}
    r = bench.gradient_roofline(info, nt=4000, s_per_grad=2.0)
    work = 2e6 * 4000 / 2.0 / 1e9
    assert r["bytes_per_cell_step"] == 236.0 and abs(r["achieved"] - 236.0 * work) < 1e-9
    assert abs(r["frac"] - 236.0 * work / peak) < 1e-12
    assert abs(r["floor_frac"] - 176.0 * work / peak) < 1e-12
    full = bench.gradient_roofline(dict(info, ckpt_interval=4000), nt=4000, s_per_grad=2.0)
    assert full["bytes_per_cell_step"] == 176.0 and full["frac"] == full["floor_frac"]
    half = bench.gradient_roofline(dict(info, ckpt_interval=4000, snap_store=1), nt=4000, s_per_grad=2.0)
    assert half["bytes_per_cell_step"] == 168.0 and half["snapshots"] == "fp16"
    assert bench.gradient_roofline(dict(info, snap_store=2), nt=4000, s_per_grad=2.0)["bytes_per_cell_step"] == 228.0
    # the final 3000 steps kept by the forward pass: 1000 recomputed steps, 176 + 60 / 4 B
    part = bench.gradient_roofline(dict(info, stored_steps=3000), nt=4000, s_per_grad=2.0)
    assert part["bytes_per_cell_step"] == 191.0 and "final 3000" in part["schedule"]
