"""Dataflow launches of a level (dataflow = 1): one launch drains the regions of all 16 groups
in group order, each region starting once the regions of earlier groups within three cells of
it are done.  Regions that touch move in group order and the others commute, so labels, cost
cache, counters and energy must equal those of the 16 group launches bit for bit (the group
launches are the ones the oracle lockstep tests check).  Every test also requires that no
region gave up waiting for a neighbour.
"""
import pytest

from synth import make_pair, workload_pair
from tests.conftest import TINY_PARAMS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _same(a, b, n_pairs=1):
    for p in range(n_pairs):
        (la, _, ca), (lb, _, cb) = a.labels(p), b.labels(p)
        assert (la.cpu().numpy() == lb.cpu().numpy()).all()
        assert (ca.cpu().numpy() == cb.cpu().numpy()).all()
    assert a.energy()[1] == b.energy()[1]


@pytest.mark.parametrize("visit", [1, 4])
def test_dataflow_equals_group_launches_middlebury(torch_cuda, visit):
    """450x375 at the paper's settings, three outer iterations (the first direct, the others
    replayed as a CUDA graph), sequential and 4-candidate visits, against group launches with
    one CTA per region and with the two-CTA cluster visits the 15 and 25 px levels take here.
    (Push-relabel counts are not compared: threads push asynchronously within a round, so the
    number of rounds varies from run to run while the minimal cut does not.)"""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 4)
    base = dict(disp_max=60.0, seed=23, candidates_per_visit=visit, work_queue=1)
    a = Stereo(pair["left"], pair["right"], cluster_visits=0, **base)
    b = Stereo(pair["left"], pair["right"], dataflow=1, **base)
    c = Stereo(pair["left"], pair["right"], **base)
    sa, sb, sc = a.iterate(3), b.iterate(3), c.iterate(3)
    assert sb.dep_waits_given_up == 0
    assert sa.maxflow_limit == 0 and sb.maxflow_limit == 0 and sc.maxflow_limit == 0
    assert sa.evals == sb.evals == sc.evals == 3 * a.evals_per_iteration()
    assert sa.accepted == sb.accepted == sc.accepted
    assert list(sa.accepted_by_kind) == list(sb.accepted_by_kind)
    _same(a, b)
    _same(c, b)


def test_dataflow_uneven_batch_and_small_cells(torch_cuda):
    """A batch of three pairs of different sizes (cell grids that are not multiples of 4, so
    the groups are uneven and the pairs' done flags are laid out one after the other), 3 px
    cells on the tiny parameters, and the launch shape changed: same bits as group launches."""
    from paper_1603_08328_gb300.lem import Stereo
    pairs = [workload_pair("tiny_96x72", 1), make_pair(7, 61, 110, 15.0, n_planes=2, n_quadrics=1),
             make_pair(8, 83, 47, 15.0, n_planes=2, n_quadrics=1)]
    params = dict(TINY_PARAMS, seed=43, cell=(3,))
    L, R = [p["left"] for p in pairs], [p["right"] for p in pairs]
    a = Stereo(L, R, **params)
    b = Stereo(L, R, dataflow=1, **params)
    c = Stereo(L, R, dataflow=1, level_threads=(128,), use_graph=0, **params)
    stats = [x.iterate(2) for x in (a, b, c)]
    assert all(s.maxflow_limit == 0 for s in stats)
    assert stats[1].dep_waits_given_up == 0 and stats[2].dep_waits_given_up == 0
    assert stats[0].accepted == stats[1].accepted == stats[2].accepted
    _same(a, b, 3)
    _same(a, c, 3)


def test_dataflow_headline_1500x1000(torch_cuda):
    """The 1500x1000 pair with FP16 images and 4-candidate visits, one outer iteration."""
    from paper_1603_08328_gb300.lem import LEM_STORE_F16, Stereo
    pair = workload_pair("large_1500x1000", 0)
    base = dict(disp_max=400.0, seed=3, store_dtype=LEM_STORE_F16, candidates_per_visit=4, work_queue=1)
    a = Stereo(pair["left"], pair["right"], **base)
    b = Stereo(pair["left"], pair["right"], dataflow=1, **base)
    sa, sb = a.iterate(1), b.iterate(1)
    assert sb.dep_waits_given_up == 0 and sa.maxflow_limit == 0 and sb.maxflow_limit == 0
    assert sa.accepted == sb.accepted
    print(f"1500x1000 iteration 0: {sa.accepted} switches, the same labels under dataflow")
    _same(a, b)


def test_dataflow_level_launches_are_timed_per_level(torch_cuda):
    """With kernel timing on, a dataflow iteration records one expansion launch per level, and
    the call's stats carry the GPU time of its iterations."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 5)
    g = Stereo(pair["left"], pair["right"], disp_max=60.0, seed=2, dataflow=1, work_queue=1)
    g.set_kernel_timing(True)
    st = g.iterate(2)
    kt = g.kernel_times()
    for lvl in range(3):
        ms, launches = kt[(lvl, "k_expand_group")]
        assert launches == 1 and ms > 0.0
    # lem_stats.ms: the GPU time of both iterations of the call, at least the last one's kernels
    assert st.ms >= sum(kt[(lvl, "k_expand_group")][0] for lvl in range(3)) > 0.0
