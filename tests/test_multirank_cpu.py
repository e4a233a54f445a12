"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.  Every
rank runs its own replica (no data-path collective); the job reports the
units of all ranks over the slowest rank's time."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is slower
    t = bench.max_over_ranks(local_ms, ws, device="cpu")
    value = bench.weak_scaling_value(ws, 1000, 4, t)
    bench.barrier(ws)
    q.put((rank, t, value))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in res:
        assert t == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)
