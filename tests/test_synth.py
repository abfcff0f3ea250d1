"""The seeded input generator (CPU): determinism, shapes, disparity ranges, the
disparity convention of the rendered pair (a left pixel u matches right pixel
u - d, Sec. 3.2, Eq. warp) and the noise level.  Both the oracle and the CUDA path
read these pairs, so a wrong convention here would go unnoticed by parity."""
import numpy as np
import pytest

from synth import WORKLOADS, batch8_pair, make_pair, random_labels, workload_pair


def test_pairs_are_seeded():
    a, b = workload_pair("tiny_96x72", 0), workload_pair("tiny_96x72", 0)
    assert (a["left"] == b["left"]).all() and (a["right"] == b["right"]).all()
    assert (a["disp"] == b["disp"]).all()
    c = workload_pair("tiny_96x72", 1)
    assert (a["left"] != c["left"]).any()


@pytest.mark.parametrize("name", ["tiny_96x72", "middlebury_450x375", "train_384x288"])
def test_shapes_and_disparity_range(name):
    cfg = WORKLOADS[name]
    for seed in range(3):
        p = workload_pair(name, seed)
        for k in ("left", "right"):
            img = p[k]
            assert img.shape == (cfg["height"], cfg["width"], 3) and img.dtype == np.uint8
            assert img.flags["C_CONTIGUOUS"]
        d = p["disp"]
        assert d.shape == (cfg["height"], cfg["width"])
        assert d.min() >= 0.0 and d.max() <= cfg["disp_max"]
        # one background plus the planar and quadric segments
        segs = p["segments"]
        assert len(segs) == 1 + cfg["n_planes"] + cfg["n_quadrics"]
        assert sum(s.kappa != 0.0 for s in segs) == cfg["n_quadrics"]


def test_first_pair_of_the_uneven_batch():
    p = batch8_pair(0)
    assert p["left"].shape == (480, 640, 3)
    assert p["disp"].min() >= 0.0 and p["disp"].max() <= 64.0


def _warp_residual(p, sign):
    """|I_L(u, v) - I_R(u + sign d(u, v), v)|_1 with I_R linearly interpolated along the
    row, at the pixels whose match lies inside the image."""
    L = p["left"].astype(np.float64)
    R = p["right"].astype(np.float64)
    D = p["disp"]
    H, W = D.shape
    v, u = np.mgrid[0:H, 0:W]
    ur = u + sign * D
    i0 = np.floor(ur).astype(np.int64)
    t = (ur - i0)[..., None]
    ok = (i0 >= 0) & (i0 + 1 < W)
    i0 = np.clip(i0, 0, W - 2)
    Ri = (1.0 - t) * R[v, i0] + t * R[v, i0 + 1]
    return np.abs(Ri - L).sum(-1)[ok]


@pytest.mark.parametrize("seed,shape", [(0, (72, 96, 15.0)), (1, (72, 96, 15.0)), (2, (375, 450, 60.0))])
def test_right_view_is_the_warp_of_the_left(seed, shape):
    """Noise-free pairs: away from occlusions the left pixel equals the right view at
    u - d up to rounding and the interpolation error of the texture (finest octave
    3 px), and the opposite sign (u + d) does not match."""
    H, W, dmax = shape
    p = make_pair(seed, H, W, dmax, n_planes=7 if W > 100 else 3, n_quadrics=3 if W > 100 else 1, sigma=0.0)
    e = _warp_residual(p, -1)
    assert np.median(e) <= 1.5
    assert np.mean(e < 6.0) >= 0.8
    assert np.median(_warp_residual(p, +1)) >= 10.0


def test_noise_level():
    """sigma = 2 gray levels, independent per view, before rounding to uint8."""
    clean = make_pair(4, 72, 96, 15.0, sigma=0.0)
    noisy = make_pair(4, 72, 96, 15.0, sigma=2.0)
    for k in ("left", "right"):
        diff = noisy[k].astype(np.float64) - clean[k].astype(np.float64)
        assert abs(diff.mean()) < 0.1
        assert 1.8 < diff.std() < 2.3
    d_l = noisy["left"].astype(np.float64) - clean["left"].astype(np.float64)
    d_r = noisy["right"].astype(np.float64) - clean["right"].astype(np.float64)
    assert abs(np.corrcoef(d_l.ravel(), d_r.ravel())[0, 1]) < 0.05


def test_random_labels():
    labs = random_labels(5, 1000, 375, 450, 60.0, slope=0.5)
    assert labs.dtype == np.float32 and labs.shape == (1000, 3)
    a, b, c = labs[:, 0].astype(np.float64), labs[:, 1].astype(np.float64), labs[:, 2].astype(np.float64)
    assert np.abs(a).max() <= 0.5 and np.abs(b).max() <= 0.5
    d_centre = a * 225.0 + b * 187.5 + c
    assert d_centre.min() >= -1e-3 and d_centre.max() <= 60.0 + 1e-3
