"""bench.py's multi-rank logic on CPU: 2 gloo ranks, barrier-bracketed timing
and the max over ranks (each GPU rank ranks its own list; there is no
collective on the data path, only this timing reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import time
    import bench
    d = bench.init_dist("gloo")
    assert d is not None and d.get_world_size() == world
    delay = 0.02 * (rank + 1)            # rank 1 is the slow one
    calls = []

    def step():
        calls.append(1)
        time.sleep(delay)
    t = bench.timed_steps(step, 3, 2, d)
    q.put((rank, t, len(calls), bench.max_over_ranks(rank + 0.5, d)))
    dist.destroy_process_group()


def test_two_rank_timing_is_max_over_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = sorted(o[1] for o in out)
    assert abs(times[0] - times[1]) < 1e-9         # every rank reports the same (max) time
    assert times[0] >= 3 * 0.04 - 1e-3             # ... which is the slow rank's K steps
    assert all(o[2] == 5 for o in out)             # W + K steps ran on each rank
    assert all(abs(o[3] - 1.5) < 1e-12 for o in out)
