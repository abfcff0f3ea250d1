"""The stripe decomposition of one pair (the multi-GPU scheme for a single image),
verified on CPU: gloo ranks, each running the oracle's expansions of the cells whose
centre cell lies in its stripe and exchanging the labels and costs of the boundary
bands after every (level, group), reproduce the single-domain run bit for bit."""
import os
import socket

import numpy as np
import pytest

from tests.conftest import TINY_PARAMS


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, left, right, params, n_iters, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle.stripes import run_stripes
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def send_recv(peer, arr):
        # the peer's band covers the rows this rank can read: its size follows from
        # the shapes both sides know, so exchange sizes first
        n_out = torch.tensor([arr.size], dtype=torch.int64)
        n_in = torch.zeros(1, dtype=torch.int64)
        reqs = [dist.isend(n_out, peer), dist.irecv(n_in, peer)]
        for r in reqs:
            r.wait()
        buf = torch.empty(int(n_in.item()), dtype=torch.float64)
        reqs = [dist.isend(torch.from_numpy(np.ascontiguousarray(arr)), peer), dist.irecv(buf, peer)]
        for r in reqs:
            r.wait()
        return buf.numpy()

    lab, cost, rows = run_stripes(rank, world, left, right, params, n_iters, send_recv)
    out.put((rank, rows, lab, cost))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, pair, params, n_iters):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("CPU-only check of the gloo path")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, pair["left"], pair["right"], params, n_iters, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def _single(pair, params, n_iters):
    import oracle
    o = oracle.Oracle(pair["left"], pair["right"], **params)
    o.init_state()
    for it in range(n_iters):
        o.iterate(it)
    return o.state()


@pytest.mark.parametrize("world", [2, 3])
def test_stripes_match_single_domain_tiny(tiny_pair, world):
    params = dict(TINY_PARAMS, n_threads=2)
    lab0, cost0 = _single(tiny_pair, params, 2)
    for rank, (t, b), lab, cost in _run(world, tiny_pair, params, 2):
        assert (lab == lab0[t:b]).all() and (cost == cost0[t:b]).all(), f"stripe {rank} rows {t}-{b}"


def test_stripes_match_single_domain_three_levels():
    """Cells 5/15/25 (stripe boundaries at multiples of 75 rows) on a 200 x 225 crop of
    the 450 x 375 scene, r' = 4, one outer iteration over 3 stripes."""
    from synth import workload_pair
    full = workload_pair("middlebury_450x375", 2)
    pair = {"left": np.ascontiguousarray(full["left"][:225, :200]),
            "right": np.ascontiguousarray(full["right"][:225, :200])}
    params = dict(gf_radius=4, disp_max=60.0, seed=4, n_threads=2)
    lab0, cost0 = _single(pair, params, 1)
    res = _run(3, pair, params, 1)
    assert [r[1] for r in res] == [(0, 75), (75, 150), (150, 225)]
    for rank, (t, b), lab, cost in res:
        assert (lab == lab0[t:b]).all() and (cost == cost0[t:b]).all(), f"stripe {rank} rows {t}-{b}"


def test_stripe_bounds():
    from oracle.stripes import stripe_bounds
    assert stripe_bounds(72, 2, [5]) == [(0, 40), (40, 72)]
    assert stripe_bounds(375, 2, [5, 15, 25]) == [(0, 150), (150, 375)]
    with pytest.raises(ValueError):
        stripe_bounds(100, 3, [5, 15, 25])
