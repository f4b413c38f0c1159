"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its
own step time and match count; the whole-job line takes the slowest rank's
time and all ranks' matches."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    step_ms = [100.0, 250.0][rank]
    matches = [1_000_000, 3_000_000][rank]
    t, v = bench.aggregate(step_ms, matches, dist, "cpu")
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, v = out[r]
        assert t == 250.0
        assert abs(v - 4_000_000 / 0.25) < 1e-6
