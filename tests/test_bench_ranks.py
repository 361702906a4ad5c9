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
