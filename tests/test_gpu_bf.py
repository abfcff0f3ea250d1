"""GPU parity of the LE-BF data term (Sec. 4: bilateral weights on the (4r'+1)^2
window instead of the guided filter) against the FP64 oracle, through the C ABI.

Tolerance: each cost is an FP32 sum of at most (4r'+1)^2 = 1681 products w * rho
with w <= 1 and rho <= (1 - alpha) tau_col + alpha tau_grad; it is summed row by row
(partial sums of at most 41 terms), so with the FP32 errors of rho (a few 1e-6
relative, from the sub-pixel warp) the error stays far below 1e-4 of the cost,
the bound the guided-filter term is held to."""
import numpy as np
import pytest

import oracle
from synth import random_labels, workload_pair
from tests.conftest import TINY_PARAMS

pytestmark = pytest.mark.gpu

BF_TINY = dict(TINY_PARAMS, data_term=1, bf_gamma=10.0, lam=20.0)


from tests.tolerance import PHI_TOL, rel_err as _rel_err, report  # noqa: E402


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.fixture(scope="module")
def tiny_bf(torch_cuda, tiny_pair):
    from paper_1603_08328_gb300.lem import Stereo
    g = Stereo(tiny_pair["left"], tiny_pair["right"], **BF_TINY)
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **BF_TINY)
    return g, o


REGIONS = [(40, 30, 15, 15), (0, 0, 10, 10), (86, 62, 10, 10), (90, 0, 6, 15), (33, 20, 7, 3), (50, 40, 1, 1),
           (0, 10, 96, 5), (20, 0, 13, 72)]


def test_bf_unary_tiny_all_regions(tiny_bf):
    g, o = tiny_bf
    K = 3
    labs = random_labels(4, len(REGIONS) * K, 72, 96, 15.0).reshape(len(REGIONS), K, 3)
    labs[0, 2] = [0.0, 0.0, 6.0]
    labs[1, 1] = [0.0, 0.0, 2.5]
    labs[2, 0] = [1.7, -0.8, -40.0]
    costs = g.unary(REGIONS, labs)
    gl, rl = [], []
    for r, lab, c in zip(REGIONS, labs, costs):
        c = c.cpu().numpy()
        for k in range(K):
            gl.append(c[k])
            rl.append(o.region_cost(*r, lab[k]))
    worst = report("LE-BF phi, ragged tiny regions", gl, rl)
    assert worst <= PHI_TOL, worst


def test_bf_unary_is_the_window_sum(tiny_bf):
    """Spot values against the per-pixel definition (lo_phi_bf), not only region_cost."""
    g, o = tiny_bf
    lab = np.array([[0.2, -0.1, 7.3]], np.float32)
    r = (10, 12, 9, 6)
    c = g.unary([r], lab[None])[0][0].cpu().numpy()
    for (yy, xx) in [(0, 0), (5, 8), (3, 4)]:
        ref = o.phi_bf(lab[0], r[0] + xx, r[1] + yy)
        assert _rel_err(c[yy, xx], ref) <= PHI_TOL


def test_bf_initial_costs(tiny_bf):
    g, o = tiny_bf
    o.init_state()
    abc, _, cost = g.labels()
    lab, ocost = o.state()
    assert (abc.cpu().numpy() == lab).all()
    worst = report("LE-BF initial cost cache", [cost.cpu().numpy()], [ocost])
    assert worst <= PHI_TOL, worst


def test_bf_unary_middlebury_shapes(torch_cuda):
    """r' = 10 (41x41 windows) on 450x375 with LE-BF: 75x75 (level-2 size), 45x45 and
    15x15 regions, interior and at the borders."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 0)
    params = dict(disp_max=60.0, seed=5, data_term=1, lam=20.0)
    g = Stereo(pair["left"], pair["right"], **params)
    o = oracle.Oracle(pair["left"], pair["right"], **params)
    regions = [(150, 120, 75, 75), (0, 0, 45, 45), (405, 300, 45, 75), (435, 360, 15, 15), (100, 200, 15, 15)]
    labs = random_labels(19, len(regions), 375, 450, 60.0).reshape(len(regions), 1, 3)
    costs = g.unary(regions, labs)
    worst = report("LE-BF phi, 450x375 regions at r' = 10", [c[0].cpu().numpy() for c in costs],
                   [o.region_cost(*r, lab[0]) for r, lab in zip(regions, labs)])
    assert worst <= PHI_TOL, worst
    st = g.iterate(1)
    assert st.maxflow_limit == 0 and st.evals == g.evals_per_iteration()
    e0 = st.energy_q
    assert g.iterate(1).energy_q <= e0
    g.close()


def test_bf_expand_groups_in_lockstep_with_oracle(tiny_pair, torch_cuda):
    """Algorithm 1 with the LE-BF data term, group by group against the oracle (same
    protocol as the LE-GF lockstep test: near-ties decided differently by the FP32 and
    FP64 costs are counted, then the oracle follows the GPU labels)."""
    from paper_1603_08328_gb300.lem import Stereo
    params = dict(BF_TINY, seed=29)
    g = Stereo(tiny_pair["left"], tiny_pair["right"], **params)
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **params)
    o.init_state()
    q_prev = g.energy()[1]
    flips = switched = 0
    per_group = []  # differing pixels of each (iteration, group), each re-synchronised
    for it in range(3):
        for grp in range(16):
            st = g.expand_group(it, 0, grp)
            acc, _ = o.expand_group(it, 0, grp)
            assert st.maxflow_limit == 0
            abc = g.labels()[0].cpu().numpy()
            lab, _ = o.state()
            per_group.append(int((abc != lab).any(axis=-1).sum()))
            flips += per_group[-1]
            switched += acc
            o.set_labels(abc)
            q = g.energy()[1]
            assert q <= q_prev
            q_prev = q
    print(f"LE-BF lockstep: {flips} differing pixels over {switched} switches")
    print(f"  differing pixels per (iteration, group) where nonzero: "
          f"{[(i, d) for i, d in enumerate(per_group) if d]}")
    assert switched > 0
    assert flips <= max(10, 0.002 * switched)


def test_bf_results_do_not_depend_on_the_launch_shape(torch_cuda):
    """LE-BF on 450x375: threads per CTA, strip rows and the two-CTA cluster visits change
    only the time.  Each raw cost and each window sum is computed by one thread with
    every operation rounded in a fixed order, so the labels and the cost cache after an
    iteration are bit-identical across the kernel instances."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("middlebury_450x375", 7)
    base = dict(disp_max=60.0, seed=19, data_term=1, lam=20.0)
    a = Stereo(pair["left"], pair["right"], **base)
    b = Stereo(pair["left"], pair["right"], level_threads=(1024, 256, 512), level_strip_rows=(8, 32, 8),
               cluster_visits=0, **base)
    a.iterate(1)
    b.iterate(1)
    (la, _, ca), (lb, _, cb) = a.labels(), b.labels()
    assert (la.cpu().numpy() == lb.cpu().numpy()).all()
    assert (ca.cpu().numpy() == cb.cpu().numpy()).all()
