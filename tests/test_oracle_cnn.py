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
