"""lem_mincut_batch_noalloc: the min-cut for callers that cannot allocate device memory.

Such callers (code inside a preallocated memory arena, a host thread that must not
call cudaMalloc because it synchronises the device) get the same cut from a fixed
scratch array in the library's device memory.  The test checks the cut against
lem_mincut_batch and, for one graph per call, against the oracle's Dinic max-flow,
and that the second call leaves the device's free memory unchanged.  This file is
collected last so a run that stops at the first failure has already run every
other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _graph(rng, w, h):
    tcap = rng.integers(0, 200000, size=(h, w, 2)).astype(np.int32)
    tcap[rng.random((h, w)) < 0.5, 0] = 0
    tcap[tcap[..., 0] > 0, 1] = 0
    ncap = rng.integers(0, 131072, size=(h, w, 4)).astype(np.int32)
    ncap[rng.random((h, w, 4)) < 0.3] = 0
    return tcap, ncap


def test_noalloc_mincut_equals_mincut_batch_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1603_08328_gb300 import lem
    from synth import workload_pair

    import oracle

    pair = workload_pair("tiny_96x72", 0)
    ref = lem.Stereo(pair["left"], pair["right"], gf_radius=2, disp_max=15.0, n_levels=1, cell=(5,),
                     k_prop=(1,), k_rand=(7,))
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    shapes = [(15, 15), (45, 45), (75, 70), (1, 16), (9, 4), (33, 7)]
    for call in range(2):
        regions = [(0, 0, w, h) for (w, h) in shapes] * (1 + call)
        graphs = [_graph(rng, w, h) for (_, _, w, h) in regions]
        tc = torch.as_tensor(np.concatenate([t.reshape(-1) for t, _ in graphs])).cuda()
        nc = torch.as_tensor(np.concatenate([c.reshape(-1) for _, c in graphs])).cuda()
        take_ref, flow_ref, st_ref = ref.mincut(regions, tc, nc)
        n = sum(w * h for (_, _, w, h) in regions)
        take = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        flow = torch.full((len(regions),), -1, dtype=torch.int64, device="cuda")
        st = torch.full((len(regions),), 99, dtype=torch.int32, device="cuda")
        p = ref.params
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lem.lem_mincut_batch_noalloc(regions, C.c_void_p(tc.data_ptr()), C.c_void_p(nc.data_ptr()),
                                          C.c_void_p(take.data_ptr()), C.c_void_p(flow.data_ptr()),
                                          C.c_void_p(st.data_ptr()), p.max_rounds, p.gr_interval,
                                          C.c_void_p(stream.cuda_stream))
        assert rc == lem.LEM_OK, lem.lem_last_error(None)
        torch.cuda.synchronize()
        if call == 1:
            # (the first call may load the library's module lazily, which places the
            # static scratch array; the second finds everything in place) no device
            # memory was taken by the call
            assert torch.cuda.mem_get_info()[0] == free_before
        # min-cut results are integers: bit-exact, as for lem_mincut_batch against the oracle
        assert (st.cpu().numpy() == 0).all() and (st_ref.cpu().numpy() == 0).all()
        assert (flow.cpu().numpy() == flow_ref.cpu().numpy()).all()
        assert (take.cpu().numpy() == take_ref.cpu().numpy()).all()
        # and the oracle's Dinic max-flow on the 45 x 45 graph of this call: flow and
        # minimal sink side bit-exact
        k = 1
        off = sum(w * h for (_, _, w, h) in regions[:k])
        w, h = regions[k][2], regions[k][3]
        f, cut = oracle.maxflow(w, h, graphs[k][0], graphs[k][1], "dinic")
        assert int(flow.cpu().numpy()[k]) == f
        assert (take.cpu().numpy()[off:off + w * h].reshape(h, w) == cut).all()
    ref.close()


def test_noalloc_rejects_more_regions_than_its_scratch_holds():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_08328_gb300 import lem
    regions = [(0, 0, 2, 2)] * (lem.LEM_NOALLOC_MAX_REGIONS + 1)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    ptr = C.c_void_p(dummy.data_ptr())
    rc = lem.lem_mincut_batch_noalloc(regions, ptr, ptr, ptr, ptr, ptr, 100, 16, None)
    assert rc == lem.LEM_ERR_ARG
    assert "LEM_NOALLOC_MAX_REGIONS" in lem.lem_last_error(None)
