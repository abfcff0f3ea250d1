"""The multi-process plumbing of bench.py (replicas: one pair per rank, barrier, max over
ranks) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, dist = bench.dist_init(world)
    assert (r, w) == (rank, world) and dist is not None
    bench.barrier(dist)
    # each replica reports its own time; the job time is the slowest rank's
    t = bench.max_over_ranks(1.0 + rank, dist)
    out.put((rank, t))
    dist.destroy_process_group()


def test_bench_replicas_max_over_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("CPU-only check of the gloo path")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 2.0), (1, 2.0)]
