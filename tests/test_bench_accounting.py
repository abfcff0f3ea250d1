"""The bench's work accounting (CPU): the counts behind `value` (pixel-label evals per
step) and the numerator of the roofline fraction (algorithmic FP32 operations per
launch), checked against independent counts and the closed forms of the region scheme
(Sec. 3.5: every candidate is evaluated on the region R, its raw cost on M = R grown by
2r', its regressions on R grown by r')."""
import numpy as np
import pytest

import bench

PAPER = dict(cell=[5, 15, 25], k_prop=[1, 2, 2], k_rand=[7, 0, 0], gf_radius=10, n_levels=3)


def _coverage(n, s):
    """How many regions along one axis contain each coordinate: the cells i with
    (i - 1) s <= u < (i + 2) s, 0 <= i < ceil(n / s)."""
    cover = np.zeros(n, np.int64)
    for i in range(-(-n // s)):
        cover[max(0, (i - 1) * s):min(n, (i + 2) * s)] += 1
    return cover


@pytest.mark.parametrize("H,W", [(375, 450), (72, 96), (1000, 1500), (101, 67)])
def test_evals_per_step_is_the_per_pixel_coverage(H, W):
    """Evals of one outer iteration = sum over pixels of (regions covering it) x
    (proposals per visit), level by level."""
    work = bench.iteration_work(H, W, PAPER)
    want = 0
    for lv, s in enumerate(PAPER["cell"]):
        n_prop = PAPER["k_prop"][lv] + PAPER["k_rand"][lv]
        want += n_prop * int(np.outer(_coverage(H, s), _coverage(W, s)).sum())
    assert sum(wk["evals"] for wk in work.values()) == want


def test_interior_pixel_gets_108_evals_per_iteration():
    """An interior pixel lies in 9 regions per level: 9 (1 + 7) + 9 x 2 + 9 x 2 = 108."""
    total = 0
    for lv, s in enumerate(PAPER["cell"]):
        n_prop = PAPER["k_prop"][lv] + PAPER["k_rand"][lv]
        total += n_prop * int(_coverage(1000, s)[500]) * int(_coverage(1000, s)[500])
    assert total == 108


def test_step_counts():
    """Evals of one outer iteration: 17 638 600 on the 450x375 pair, 160 252 300 on the
    1500x1000 headline pair (the library's lem_evals_per_iteration reports the same)."""
    assert sum(wk["evals"] for wk in bench.iteration_work(375, 450, PAPER).values()) == 17638600
    assert sum(wk["evals"] for wk in bench.iteration_work(1000, 1500, PAPER).values()) == 160252300


@pytest.mark.parametrize("s,per_eval", [(5, 666), (15, 223), (25, 165)])
def test_interior_flops_per_eval(s, per_eval):
    """Interior region R = 3s x 3s at r' = 10: 30 |M| + 44 |R + r'| + 24 |R| per candidate,
    i.e. about 666 / 223 / 165 FP32 operations per pixel-label eval."""
    R = 3 * s
    f = bench.algorithmic_flops(2000, 2000, 10, 500, 500, R, R)
    assert f == 30 * (R + 40) ** 2 + 44 * (R + 20) ** 2 + 24 * R * R
    assert abs(f / (R * R) - per_eval) < 1.0


def test_flops_clip_at_the_border():
    """At the image corner M and the regression range are clipped to the image."""
    s, r = 25, 10
    f = bench.algorithmic_flops(375, 450, r, 0, 0, 2 * s, 2 * s)
    assert f == 30 * (2 * s + 2 * r) ** 2 + 44 * (2 * s + r) ** 2 + 24 * (2 * s) ** 2


def test_groups_are_disjoint_and_cover_every_region():
    """Regions of one group never overlap (cells of a group are 4 apart, regions 3 cells
    wide), and the 16 groups hold every cell's region once."""
    H, W, s = 375, 450, 15
    groups = bench.region_geometry(H, W, s)
    assert sum(len(v) for v in groups.values()) == (-(-H // s)) * (-(-W // s))
    for regs in groups.values():
        owner = np.zeros((H, W), np.int64)
        for (x0, y0, w, h) in regs:
            owner[y0:y0 + h, x0:x0 + w] += 1
        assert owner.max() <= 1


def test_bf_flops_interior():
    """LE-BF: 30 per raw cost over M and one multiply-add per window pixel of each output
    pixel; in the interior every window is (4r' + 1)^2."""
    s, r = 15, 10
    R = 3 * s
    f = bench.bf_flops(2000, 2000, r, 500, 500, R, R)
    assert f == 30 * (R + 4 * r) ** 2 + 2 * (4 * r + 1) ** 2 * R * R
