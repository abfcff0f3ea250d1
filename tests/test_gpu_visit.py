"""GPU parity of the batched-visit path (candidates_per_visit >= 2): the warp data term
(one warp per region and candidate, exact fixed-point window sums) and the cut
launch that makes the visit's moves, against the FP64 oracle through the C ABI.

lem_unary_batch on a handle with batched visits runs the same warp data term, so the
data-term checks below call it on such handles.  Tolerances are those of the data
term (tests/tolerance.py); labels are compared group by group as in the other
lockstep tests, with every differing pixel counted and the oracle re-synchronised.
"""
import numpy as np
import pytest

import oracle
from synth import random_labels, workload_pair
from tests.conftest import TINY_PARAMS
from tests.tolerance import PHI_TOL, PHI_TOL_16, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _unary_check(g, o, regions, labs, label):
    costs = g.unary(regions, labs)
    gl, rl = [], []
    for r, lab, c in zip(regions, labs, costs):
        c = c.cpu().numpy()
        for k in range(lab.shape[0]):
            gl.append(c[k])
            rl.append(o.region_cost(*r, lab[k]))
    return report(label, gl, rl)


def test_warp_data_term_tiny_ragged_regions(torch_cuda, tiny_pair):
    """r' = 2: regions of every shape the 5 and 15 px levels make, corners, a full-width
    strip, 1x1, a steep plane whose matches leave the image."""
    from paper_1603_08328_gb300.lem import Stereo
    params = dict(TINY_PARAMS, candidates_per_visit=4, split_visits=1)
    g = Stereo(tiny_pair["left"], tiny_pair["right"], **params)
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    regions = [(40, 30, 15, 15), (0, 0, 10, 10), (86, 62, 10, 10), (90, 0, 6, 15), (0, 57, 15, 15), (33, 20, 7, 3),
               (50, 40, 1, 1), (0, 10, 96, 5), (20, 0, 13, 72), (30, 15, 45, 45), (51, 27, 45, 45)]
    K = 3
    labs = random_labels(31, len(regions) * K, 72, 96, 15.0).reshape(len(regions), K, 3)
    labs[0, 2] = [0.0, 0.0, 6.0]
    labs[1, 1] = [0.0, 0.0, 2.5]
    labs[2, 0] = [1.7, -0.8, -40.0]
    worst = _unary_check(g, o, regions, labs, "warp phi, tiny ragged regions")
    assert worst <= PHI_TOL, worst


def test_warp_data_term_middlebury_shapes(torch_cuda):
    """r' = 10 (41x41 windows) on 450x375: 75x75 (four M columns per lane), 45x45 (three),
    15x15 (two), clipped at every border."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 0)
    params = dict(disp_max=60.0, seed=4, candidates_per_visit=4, split_visits=1)
    g = Stereo(pair["left"], pair["right"], **params)
    o = oracle.Oracle(pair["left"], pair["right"], disp_max=60.0, seed=4)
    regions = [(150, 120, 75, 75), (0, 0, 50, 50), (400, 300, 50, 75), (200, 45, 45, 45), (435, 360, 15, 15),
               (100, 200, 15, 15), (0, 180, 15, 15), (375, 0, 75, 45)]
    labs = random_labels(9, len(regions) * 2, 375, 450, 60.0).reshape(len(regions), 2, 3)
    labs[3, 1] = [0.0, 0.0, 17.0]
    worst = _unary_check(g, o, regions, labs, "warp phi, 450x375 regions at r' = 10")
    assert worst <= PHI_TOL, worst


def test_warp_data_term_fp16_1500x1000(torch_cuda):
    from paper_1603_08328_gb300.lem import LEM_STORE_F16, Stereo
    pair = workload_pair("large_1500x1000", 0)
    params = dict(disp_max=400.0, candidates_per_visit=4, split_visits=1)
    g = Stereo(pair["left"], pair["right"], store_dtype=LEM_STORE_F16, **params)
    o = oracle.Oracle(pair["left"], pair["right"], disp_max=400.0)
    regions = [(700, 500, 15, 15), (300, 620, 45, 45), (600, 400, 75, 75), (0, 0, 50, 50), (1460, 300, 40, 75),
               (20, 955, 75, 45)]
    labs = random_labels(17, 2 * len(regions), 1000, 1500, 400.0, 0.3).reshape(len(regions), 2, 3)
    worst = _unary_check(g, o, regions, labs, "warp phi, 1500x1000 FP16")
    assert worst <= PHI_TOL_16, worst


def test_batched_visits_in_lockstep_with_oracle_middlebury(torch_cuda):
    """One outer iteration of the batched schedule (4 candidates per visit) on the 450x375
    pair at the paper's settings, level by level and group by group: the GPU and the oracle
    start each group from the same labels, draw the same candidates and make the same moves.
    Every pixel whose label differs is counted (a near-tie the FP32 and FP64 data terms decide
    differently) and the oracle is re-synchronised; the counts per group are the result, the
    bound only a guard."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 2)
    params = dict(disp_max=60.0, seed=29, candidates_per_visit=4, split_visits=1)
    g = Stereo(pair["left"], pair["right"], **params)
    o = oracle.Oracle(pair["left"], pair["right"], visit=4, disp_max=60.0, seed=29)
    o.init_state()
    q_prev = g.energy()[1]
    per_group, switched = [], 0
    for lvl in range(3):
        for grp in range(16):
            st = g.expand_group(0, lvl, grp)
            acc, _ = o.expand_group(0, lvl, grp)
            assert st.maxflow_limit == 0
            abc = g.labels()[0].cpu().numpy()
            lab, _ = o.state()
            per_group.append(int((abc != lab).any(axis=-1).sum()))
            switched += acc
            o.set_labels(abc)
            q = g.energy()[1]
            assert q <= q_prev
            q_prev = q
    flips = sum(per_group)
    print(f"batched-visit lockstep 450x375: {flips} differing pixels over {switched} switches; per (level, group) "
          f"{per_group}")
    assert switched > 0
    assert flips <= max(10, 0.002 * switched)


def test_batched_visit_launch_shape_and_graph_do_not_change_results(torch_cuda):
    """The cut CTA's size, the relabel interval and CUDA-graph replay change only the time:
    labels, cost cache and energy after two iterations are bit-identical."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 3)
    base = dict(disp_max=60.0, seed=9, candidates_per_visit=4, split_visits=1)
    a = Stereo(pair["left"], pair["right"], **base)
    b = Stereo(pair["left"], pair["right"], level_threads=(32, 1024, 128), level_gr_interval=(64, 8, 32), **base)
    c = Stereo(pair["left"], pair["right"], level_threads=(256, 64, 1024), use_graph=0, **base)
    for x in (a, b, c):
        st = x.iterate(2)
        assert st.maxflow_limit == 0 and st.evals == 2 * x.evals_per_iteration()
    (la, _, ca), (lb, _, cb), (lc, _, cc) = (x.labels() for x in (a, b, c))
    for l2, c2 in ((lb, cb), (lc, cc)):
        assert (la.cpu().numpy() == l2.cpu().numpy()).all()
        assert (ca.cpu().numpy() == c2.cpu().numpy()).all()
    assert a.energy()[1] == b.energy()[1] == c.energy()[1]
