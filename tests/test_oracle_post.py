"""Pins of the right-view and post-processing reference (oracle/postproc.py)."""
import numpy as np
import pytest

from oracle import postproc as pp


def test_mirrored_planes_give_the_right_view_disparity():
    """A plane found at mirrored column u' = W - 1 - u, converted, gives the same
    disparity at right pixel u."""
    rng = np.random.default_rng(0)
    H, W = 7, 11
    abc_m = rng.normal(size=(H, W, 3))
    right = pp.mirror_planes_to_right(abc_m)
    v, u = np.mgrid[0:H, 0:W]
    d_right = right[..., 0] * u + right[..., 1] * v + right[..., 2]
    um = W - 1 - u
    d_m = abc_m[v, um, 0] * um + abc_m[v, um, 1] * v + abc_m[v, um, 2]
    assert np.allclose(d_right, d_m, atol=1e-12)


def test_lr_check_of_a_constant_disparity():
    """d = 5 in both views: pixels whose match falls inside the right image are consistent."""
    H, W = 4, 12
    dL = np.full((H, W), 5.0, np.float32)
    dR = np.full((H, W), 5.0, np.float32)
    ok = pp.lr_check(dL, dR)
    assert (ok[:, 5:]).all() and not ok[:, :5].any()
    # a right view that disagrees by more than one pixel invalidates everything
    assert not pp.lr_check(dL, dR + 1.5).any()
    assert pp.lr_check(dL, dR + 1.0)[:, 5:].all()


def test_lr_check_rounds_the_match_half_to_even():
    dL = np.array([[2.5, 0, 0, 0, 0]], np.float32)
    dR = np.array([[0, 0, 2.5, 0, 0]], np.float32)
    dR2 = np.array([[0, 2.5, 0, 0, 0]], np.float32)
    # u = 4: 4 - 2.5 = 1.5 -> 2; u = 0 has match -2.5 -> outside
    dL4 = np.array([[0, 0, 0, 0, 2.5]], np.float32)
    assert pp.lr_check(dL4, dR)[0, 4] and not pp.lr_check(dL4, dR2)[0, 4]
    assert not pp.lr_check(dL, dR)[0, 0]


def test_fill_takes_the_background_plane():
    """A gap between a foreground (d = 20) and a background (d = 5 + 0.1 u) pixel takes
    the background plane evaluated at the gap pixel; at the image border only one side."""
    H, W = 1, 9
    abc = np.zeros((H, W, 3), np.float32)
    abc[0, :3] = (0, 0, 20)
    abc[0, 6:] = (0.1, 0, 5)
    valid = np.ones((H, W), bool)
    valid[0, 3:6] = False
    valid[0, 8] = False
    d = pp.fill_invalid(abc, valid)
    for x in (3, 4, 5):
        assert d[0, x] == np.float32(np.float32(0.1) * np.float32(x) + np.float32(5))
    assert d[0, 8] == np.float32(np.float32(0.1) * np.float32(8) + np.float32(5))
    assert (d[0, :3] == 20).all()


def test_weighted_median_with_equal_weights_is_the_lower_median():
    rng = np.random.default_rng(1)
    H, W = 9, 9
    disp = rng.normal(size=(H, W))
    left = np.full((H, W, 3), 100.0)
    valid = np.ones((H, W), bool)
    valid[4, 4] = False
    out = pp.weighted_median(disp, valid, left, radius=2)
    win = np.sort(disp[2:7, 2:7].ravel())
    assert out[4, 4] == win[(win.size + 1) // 2 - 1]
    assert (out[valid] == disp[valid]).all()


def test_weighted_median_follows_the_colour_weights():
    """One pixel of the window shares the centre's colour, the rest are far: its value
    wins when its weight exceeds the rest; every output is a valid weighted median."""
    H, W = 5, 5
    disp = np.arange(25, dtype=np.float64).reshape(H, W)
    left = np.zeros((H, W, 3))
    left[2, 2] = left[0, 0] = 200.0
    valid = np.ones((H, W), bool)
    valid[2, 2] = False
    out = pp.weighted_median(disp, valid, left, radius=2, gamma=10.0)
    w = np.exp(-np.abs(left - left[2, 2]).sum(-1) / 10.0)
    assert pp.is_weighted_median(out[2, 2], disp.ravel(), w.ravel())
    # the two bright pixels (values 0 and 12) hold almost all the weight: the lower wins
    assert out[2, 2] == 0.0


@pytest.mark.parametrize("edge", ["last row", "last column", "first row", "first column"])
def test_weighted_median_window_reaches_the_radius(edge):
    """Rule 3's window holds r rows and columns on every side of the pixel ((2r + 1)^2,
    r = 2 here).  With equal weights (one colour) and 25 values (12 zeros, 8 twos and five
    ones on one edge of the window) the lower median is 1; without that edge it would be 0."""
    H = W = 12
    r, y, x = 2, 5, 5
    left = np.full((H, W, 3), 80, np.uint8)
    valid = np.ones((H, W), bool)
    valid[y, x] = False
    win = np.full((5, 5), 2.0)
    sl = {"last row": np.s_[4, :], "last column": np.s_[:, 4], "first row": np.s_[0, :],
          "first column": np.s_[:, 0]}[edge]
    win[sl] = 1.0
    rest = np.argwhere(win == 2.0)[:12]
    win[rest[:, 0], rest[:, 1]] = 0.0
    disp = np.full((H, W), 9.0)
    disp[y - r:y + r + 1, x - r:x + r + 1] = win
    out = pp.weighted_median(disp, valid, left, radius=r, gamma=10.0)
    assert out[y, x] == 1.0
    assert (out[valid] == disp[valid]).all()
