"""Images smaller than a region, a cell or a matching window: the degenerate sizes of the
method down to one regression window (5 x 5 pixels at r' = 2, the smallest image lem_create
takes): cell grids of 1 x 1 and 2 x 3 cells, regions and matching windows clipped on every side.
Each size runs Algorithm 1 group by group in lockstep with the FP64 oracle, with three grid
levels, and the dataflow level launch must give the labels of the group launches there as well.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _pair(seed, H, W, shift=2):
    """A textured left image and the right image that sees it shifted by `shift` pixels."""
    rng = np.random.default_rng(seed)
    wide = rng.integers(0, 256, size=(H, W + shift, 3), dtype=np.uint8)
    return np.ascontiguousarray(wide[:, shift:]), np.ascontiguousarray(wide[:, :W])


SIZES = [(5, 5), (5, 40), (6, 9), (12, 5), (17, 33), (30, 80)]
PARAMS = dict(gf_radius=2, disp_max=6.0, cell=(2, 5, 9), seed=17)


@pytest.mark.parametrize("H,W", SIZES)
def test_small_images_in_lockstep_with_oracle(torch_cuda, H, W):
    from paper_1603_08328_gb300.lem import Stereo
    L, R = _pair(H * 100 + W, H, W)
    g = Stereo(L, R, **PARAMS)
    o = oracle.Oracle(L, R, **PARAMS)
    o.init_state()
    q_prev = g.energy()[1]
    flips = switched = 0
    for it in range(2):
        for lvl in range(3):
            for grp in range(16):
                st = g.expand_group(it, lvl, grp)
                acc, _ = o.expand_group(it, lvl, grp)
                assert st.maxflow_limit == 0
                abc = g.labels()[0].cpu().numpy()
                lab, _ = o.state()
                flips += int((abc != lab).any(axis=-1).sum())
                switched += acc
                o.set_labels(abc)
                q = g.energy()[1]
                assert q <= q_prev
                q_prev = q
    print(f"{H}x{W}: {flips} differing pixels over {switched} switches")
    assert flips <= max(2, 0.002 * switched)


@pytest.mark.parametrize("H,W", SIZES)
def test_small_images_dataflow_equals_group_launches(torch_cuda, H, W):
    from paper_1603_08328_gb300.lem import Stereo
    L, R = _pair(H * 100 + W + 1, H, W)
    a = Stereo(L, R, **PARAMS)
    b = Stereo(L, R, dataflow=1, work_queue=1, **PARAMS)
    sa, sb = a.iterate(3), b.iterate(3)
    assert sa.maxflow_limit == 0 and sb.maxflow_limit == 0 and sb.dep_waits_given_up == 0
    assert sa.accepted == sb.accepted
    assert (a.labels()[0].cpu().numpy() == b.labels()[0].cpu().numpy()).all()
    assert a.energy()[1] == b.energy()[1]
