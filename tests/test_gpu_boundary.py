"""The boundary's general forms on the GPU: images of every element type and layout that
lem_image describes, and batch calls whose regions name their pair (lem_region.img).

Images: the method works on 8-bit colours, so a handle created from the same colours as
float32 / float16 / bfloat16 values, with an alpha channel, or with padded rows, must be
the handle of the packed uint8 image bit for bit (labels and energy after an outer
iteration).  Batch calls: the data term and the graph of regions of pair 1 of a batch
handle against the FP64 oracle of that pair, in calls that mix regions of both pairs.
"""
import numpy as np
import pytest

import oracle
from synth import make_pair, random_labels, workload_pair
from tests.conftest import TINY_PARAMS
from tests.tolerance import PHI_TOL, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _run(left, right):
    from paper_1603_08328_gb300.lem import Stereo
    g = Stereo(left, right, **dict(TINY_PARAMS, seed=19))
    st = g.iterate(1)
    assert st.maxflow_limit == 0
    out = g.labels()[0].cpu().numpy(), g.energy()[1]
    g.close()
    return out


def test_image_layouts_give_the_packed_rgb8_handle(torch_cuda):
    torch = torch_cuda
    pair = workload_pair("tiny_96x72", 2)
    L, R = pair["left"], pair["right"]
    H, W = L.shape[:2]
    ref_lab, ref_q = _run(L, R)
    rng = np.random.default_rng(3)

    def rgba(x):
        return np.concatenate([x, rng.integers(0, 256, size=(H, W, 1), dtype=np.uint8)], axis=2)

    def padded(x, dtype):
        t = torch.zeros((H, W + 7, 3), dtype=dtype, device="cuda")
        t[:, :W] = torch.as_tensor(x).to(dtype).cuda()
        return t[:, :W]          # strides ((W + 7) * 3, 3, 1)

    variants = {
        "host float32": (L.astype(np.float32), R.astype(np.float32)),
        "host float16": (L.astype(np.float16), R.astype(np.float16)),
        "host float32 off the integers (rounded)": (L.astype(np.float32) + 0.3, R.astype(np.float32) - 0.4),
        "host uint8 RGBA": (rgba(L), rgba(R)),
        "device uint8 RGBA": (torch.as_tensor(rgba(L)).cuda(), torch.as_tensor(rgba(R)).cuda()),
        "device float32 RGBA": (torch.as_tensor(rgba(L).astype(np.float32)).cuda(),
                                torch.as_tensor(rgba(R).astype(np.float32)).cuda()),
        "device bfloat16, padded rows": (padded(L, torch.bfloat16), padded(R, torch.bfloat16)),
        "device uint8, padded rows": (padded(L, torch.uint8), padded(R, torch.uint8)),
    }
    for name, (l, r) in variants.items():
        lab, q = _run(l, r)
        assert (lab == ref_lab).all(), name
        assert q == ref_q, name


def test_right_view_from_float_images(torch_cuda):
    """The right-view handle (mirrored pair) from float32 images equals the one from uint8."""
    from paper_1603_08328_gb300.lem import Stereo
    pair = workload_pair("tiny_96x72", 3)
    a = Stereo(pair["left"], pair["right"], view="right", **TINY_PARAMS)
    b = Stereo(pair["left"].astype(np.float32), pair["right"].astype(np.float32), view="right", **TINY_PARAMS)
    a.iterate(1)
    b.iterate(1)
    assert (a.labels()[0].cpu().numpy() == b.labels()[0].cpu().numpy()).all()


def test_batch_calls_take_each_regions_pair(torch_cuda):
    from paper_1603_08328_gb300.lem import LemError, Stereo
    p0 = workload_pair("tiny_96x72", 0)
    p1 = make_pair(6, 61, 110, 15.0, n_planes=2, n_quadrics=1)
    params = dict(TINY_PARAMS, seed=13)
    g = Stereo([p0["left"], p1["left"]], [p0["right"], p1["right"]], **params)
    g.iterate(1)                                            # realistic current labels
    oracles = [oracle.Oracle(p["left"], p["right"], **params) for p in (p0, p1)]
    states = []
    for b, o in enumerate(oracles):
        abc, _, cost = g.labels(b)
        lab, c64 = abc.cpu().numpy(), cost.cpu().numpy().astype(np.float64)
        o.put_state(lab, c64)
        states.append((lab, c64))
    # data term: regions of both pairs in one call, the pair-1 ones crossing its borders
    regions = [(30, 20, 15, 15, 1), (40, 30, 15, 15, 0), (95, 46, 15, 15, 1), (0, 0, 10, 10, 1),
               (86, 62, 10, 10, 0), (0, 50, 110, 11, 1), (7, 3, 1, 1, 1)]
    K = 3
    labs = random_labels(8, len(regions) * K, 61, 110, 15.0).reshape(len(regions), K, 3)
    costs = g.unary(regions, labs)
    got, ref = [], []
    for r, lab, c in zip(regions, labs, costs):
        c = c.cpu().numpy()
        for k in range(K):
            got.append(c[k])
            ref.append(oracles[r[4]].region_cost(*r[:4], lab[k]))
    worst = report("phi, regions of two pairs in one call", got, ref)
    assert worst <= PHI_TOL
    # graph: against the labels of each region's own pair
    regions = [(35, 25, 15, 15, 1), (20, 10, 15, 15, 0), (95, 50, 15, 11, 1), (0, 0, 9, 7, 1)]
    rng = np.random.default_rng(5)
    alpha = np.stack([states[r[4]][0][r[1] + 1, r[0] + 1] + np.float32([0.01, -0.01, 0.4]) * rng.standard_normal(3)
                      for r in regions]).astype(np.float32)
    ca = [c[0] for c in g.unary(regions, alpha[:, None, :])]
    tc, nc, ct = (x.cpu().numpy() for x in g.pairwise(regions, alpha, ca))
    off = exact = total = 0
    for i, r in enumerate(regions):
        n = r[2] * r[3]
        lab, c64 = states[r[4]]
        gref = oracles[r[4]].build_graph(*r[:4], alpha[i], lab, c64, ca[i].cpu().numpy().astype(np.float64))
        gt = tc[2 * off:2 * (off + n)].reshape(r[3], r[2], 2)
        gn = nc[4 * off:4 * (off + n)].reshape(r[3], r[2], 4)
        assert np.abs(gn - gref["ncap"]).max() <= 3
        du = (gt[..., 0] - gt[..., 1]) - (gref["tcap"][..., 0] - gref["tcap"][..., 1])
        assert np.abs(du).max() <= 12
        assert abs(int(ct[i]) - gref["const"]) <= 12 * n
        exact += (gn == gref["ncap"]).sum() + (du == 0).sum()
        total += gn.size + du.size
        off += n
    assert exact / total > 0.9, exact / total
    # a region outside its own pair's image, a pair index out of range, a centre cell
    # outside its region
    one = np.zeros((1, 1, 3), np.float32)
    for bad in [(101, 0, 10, 10, 1), (0, 0, 5, 5, 2), (0, 0, 5, 5, -1), (10, 10, 9, 9, 0, 0, 0, 3, 3)]:
        with pytest.raises(LemError):
            g.unary([bad], one)
    # a valid centre cell is accepted and changes nothing
    c1 = g.unary([(30, 20, 15, 15, 1, 35, 25, 5, 5)], labs[:1, :1])[0].cpu().numpy()
    c2 = g.unary([(30, 20, 15, 15, 1)], labs[:1, :1])[0].cpu().numpy()
    assert (c1 == c2).all()
