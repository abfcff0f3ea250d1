"""Pins of the FP64 network reference: scipy correlation and finite differences."""
import numpy as np
import pytest

from oracle import cnn


def test_conv3x3_is_zero_padded_correlation():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(9, 11, 3))
    w = rng.normal(size=(3, 3, 3, 2))
    y = cnn.conv3x3(x, w)
    for o in range(2):
        ref = sum(scipy_signal.correlate2d(x[..., c], w[..., c, o], mode="same", boundary="fill")
                  for c in range(3))
        assert np.allclose(y[..., o], ref, atol=1e-12)


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    layers = [(7, 4), (4, 4), (4, 3)]
    params = [(rng.normal(scale=0.4, size=(3, 3, ci, co)), rng.normal(scale=0.1, size=co)) for ci, co in layers]
    x = rng.normal(size=(6, 5, 7))
    target = rng.normal(size=(6, 5, 3))
    scale = np.array([1.0, 2.0, 0.5])

    def loss_of(ps):
        out, _, _ = cnn.forward(ps, x)
        return cnn.l1_loss(out, target, scale)[0]

    out, acts, pre = cnn.forward(params, x)
    _, dout = cnn.l1_loss(out, target, scale)
    grads = cnn.backward(params, acts, pre, dout)
    eps = 1e-6
    for li in range(len(params)):
        w, b = params[li]
        for idx in [(0, 0, 0, 0), (1, 2, 3, 1), (2, 1, 0, 2)]:
            if any(i >= s for i, s in zip(idx, w.shape)):
                continue
            wp = w.copy(); wp[idx] += eps
            wm = w.copy(); wm[idx] -= eps
            pp = list(params); pp[li] = (wp, b)
            pm = list(params); pm[li] = (wm, b)
            fd = (loss_of(pp) - loss_of(pm)) / (2 * eps)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-4, abs=1e-7)
        bp = b.copy(); bp[0] += eps
        bm = b.copy(); bm[0] -= eps
        pp = list(params); pp[li] = (w, bp)
        pm = list(params); pm[li] = (w, bm)
        fd = (loss_of(pp) - loss_of(pm)) / (2 * eps)
        assert grads[li][1][0] == pytest.approx(fd, rel=1e-4, abs=1e-7)


def test_input_gradient_by_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(5, 4, 3))
    w = rng.normal(size=(3, 3, 3, 2))
    dy = rng.normal(size=(5, 4, 2))
    dx = cnn.conv3x3_grad_input(dy, w)
    eps = 1e-6
    for idx in [(0, 0, 0), (2, 3, 1), (4, 1, 2)]:
        xp = x.copy(); xp[idx] += eps
        xm = x.copy(); xm[idx] -= eps
        fd = ((cnn.conv3x3(xp, w) * dy).sum() - (cnn.conv3x3(xm, w) * dy).sum()) / (2 * eps)
        assert dx[idx] == pytest.approx(fd, rel=1e-6)


def test_quarter_features_and_targets_of_a_global_plane():
    """A single plane d = a u + b v + c: the 4x4 block mean of d is d at the block centre
    (d is linear), the block means of a, b are a, b, and constant colours stay constant."""
    H, W, dmax = 16, 20, 40.0
    a, b, c = 0.3, -0.2, 9.0
    lab = np.broadcast_to(np.array([a, b, c]), (H, W, 3)).copy()
    left = np.full((H, W, 3), 51.0)
    right = np.full((H, W, 3), 102.0)
    x = cnn.quarter_features(left, right, lab, dmax)
    t = cnn.quarter_targets(lab, dmax)
    for V in range(H // 4):
        for U in range(W // 4):
            d_centre = a * (4 * U + 1.5) + b * (4 * V + 1.5) + c
            assert np.allclose(x[V, U, :3], 0.2) and np.allclose(x[V, U, 3:6], 0.4)
            assert x[V, U, 6] == pytest.approx(d_centre / dmax, rel=1e-12)
            assert t[V, U] == pytest.approx([d_centre / dmax, a, b], rel=1e-12)


def test_upsampling_reproduces_a_global_plane():
    """Bilinear interpolation of a linear function is exact: (d/dmax, a, b) sampled from one
    plane at the quarter-cell centres gives that plane back at every pixel between the first
    and last centres (and a, b everywhere)."""
    H, W, dmax = 23, 30, 50.0
    a, b, c = -0.15, 0.4, 12.5
    H4, W4 = (H + 3) // 4, (W + 3) // 4
    y = np.zeros((H4, W4, 3))
    for V in range(H4):
        for U in range(W4):
            y[V, U] = ((a * (4 * U + 1.5) + b * (4 * V + 1.5) + c) / dmax, a, b)
    out = cnn.upsample_planes(y, H, W, dmax)
    assert np.allclose(out[..., 0], a) and np.allclose(out[..., 1], b)
    inner = out[2:4 * (H4 - 1) + 2, 2:4 * (W4 - 1) + 2]
    assert np.allclose(inner[..., 2], c, atol=1e-9)


def test_round_bf16_ties_to_even_and_matches_torch():
    """bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie that goes to the even 1.0,
    1 + 3 * 2^-8 a tie that goes up to 1 + 2^-6, and torch's CPU conversion agrees on
    random values over many binades."""
    assert cnn.round_bf16([1.0 + 2.0 ** -8])[0] == 1.0
    assert cnn.round_bf16([1.0 + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6
    assert cnn.round_bf16([1.0 + 2.0 ** -8 + 2.0 ** -20])[0] == 1.0 + 2.0 ** -7
    assert cnn.round_bf16([-3.0])[0] == -3.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = (rng.normal(size=4000) * np.exp2(rng.integers(-30, 30, size=4000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert (cnn.round_bf16(x) == ref).all()


def test_bf16_storage_model_is_the_rounded_network():
    """store='bf16' is the plain network applied to rounded weights and inputs when every
    activation is already a bfloat16 value (then the stored roundings change nothing)."""
    rng = np.random.default_rng(6)
    layers = [(7, 4), (4, 3)]
    params = [(rng.normal(size=(3, 3, ci, co)), rng.normal(size=co)) for ci, co in layers]
    x = rng.normal(size=(5, 6, 7))
    out_s, acts_s, _ = cnn.forward(params, x, store="bf16")
    rp = [(cnn.round_bf16(w), b) for w, b in params]
    h1 = np.maximum(cnn.conv3x3(cnn.round_bf16(x), rp[0][0], rp[0][1]), 0.0)
    assert (acts_s[1] == cnn.round_bf16(h1)).all()
    assert np.allclose(out_s, cnn.conv3x3(cnn.round_bf16(h1), rp[1][0], rp[1][1]), rtol=0, atol=1e-12)


def test_targets_clamp_steep_slopes():
    """Mean slopes beyond +-1 are clamped; the disparity channel is not."""
    lab = np.zeros((4, 4, 3))
    lab[..., 0] = 3.0
    lab[..., 1] = -0.5
    t = cnn.quarter_targets(lab, 10.0)
    assert t[0, 0, 1] == 1.0 and t[0, 0, 2] == -0.5
    # d = 3 u - 0.5 v averaged over the block: 3 * 1.5 - 0.5 * 1.5 = 3.75, over dmax = 10
    assert t[0, 0, 0] == pytest.approx(0.375)


def test_adam_closed_forms():
    """Adam (Kingma and Ba 2015): on the first step the bias-corrected moments are g and g^2,
    so every parameter moves by lr g / (|g| + eps), i.e. by lr against the sign of its
    gradient; a second step with the same gradient moves it by lr again; a zero gradient
    leaves it in place; and the moments follow their recurrences."""
    rng = np.random.default_rng(0)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    g[:5] = 0.0
    z = np.zeros(50)
    w1, m1, v1 = cnn.adam_step(w, g, z, z, 1, 1e-3)
    assert np.allclose(w1 - w, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert (w1[:5] == w[:5]).all()
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    w2, m2, v2 = cnn.adam_step(w1, g, m1, v1, 2, 1e-3)
    nz = g != 0
    assert np.allclose((w2 - w1)[nz], -1e-3 * np.sign(g[nz]), rtol=1e-6, atol=0)
    assert np.allclose(m2, 0.19 * g) and np.allclose(v2, (0.001 * 0.999 + 0.001) * g * g)
    # a gradient that changes sign: the first moment carries the old direction
    w3, _, _ = cnn.adam_step(w1, -g, m1, v1, 2, 1e-3)
    mh = (0.9 * 0.1 * g - 0.1 * g) / (1 - 0.81)
    vh = (0.999 * 0.001 + 0.001) * g * g / (1 - 0.999 ** 2)
    assert np.allclose(w3 - w1, -1e-3 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-9, atol=1e-15)
