"""FP64 reference of the plane-proposal network (test infrastructure only).

The network maps the stereo pair and the current label map, at quarter
resolution, to per-pixel plane proposals: 6 layers of 3x3 convolutions (zero
padding, stride 1), 32 channels, ReLU after all but the last, input channels
(left RGB, right RGB, disparity), output (d, a, b).  Only the tests use this
module; it shares no code with the CUDA kernels.

Layouts: activations are (H, W, C); weights of a layer are (3, 3, Cin, Cout)
(kernel row, kernel column, input channel, output channel); y = x * w + bias
with y[v, u, o] = sum_{i,j,c} x[v + i - 1, u + j - 1, c] w[i, j, c, o].

Parity pins: tests/test_oracle_cnn.py (finite differences, scipy correlation).
"""
from __future__ import annotations

import numpy as np

LAYERS = [(7, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 3)]


def conv3x3(x, w, b=None):
    """Zero-padded 3x3 convolution (cross-correlation), x (H, W, Cin), w (3, 3, Cin, Cout)."""
    H, W, _ = x.shape
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    y = np.zeros((H, W, w.shape[3]))
    for i in range(3):
        for j in range(3):
            y += xp[i:i + H, j:j + W] @ w[i, j]
    if b is not None:
        y += b
    return y


def conv3x3_grad_input(dy, w):
    """d loss / d x of conv3x3 given d loss / d y."""
    H, W, _ = dy.shape
    dyp = np.zeros((H + 2, W + 2, dy.shape[2]))
    dyp[1:-1, 1:-1] = dy
    dx = np.zeros((H, W, w.shape[2]))
    # x[v, u] contributes to y[v - i + 1, u - j + 1] through w[i, j]
    for i in range(3):
        for j in range(3):
            dx += dyp[2 - i:2 - i + H, 2 - j:2 - j + W] @ w[i, j].T
    return dx


def conv3x3_grad_weight(x, dy):
    """d loss / d w (3, 3, Cin, Cout) and d loss / d bias."""
    H, W, _ = x.shape
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    dw = np.zeros((3, 3, x.shape[2], dy.shape[2]))
    for i in range(3):
        for j in range(3):
            dw[i, j] = xp[i:i + H, j:j + W].reshape(-1, x.shape[2]).T @ dy.reshape(-1, dy.shape[2])
    return dw, dy.sum(axis=(0, 1))


def forward(params, x):
    """params: list of (w, b); returns the output and the per-layer inputs/pre-activations."""
    acts, pre = [x], []
    h = x
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts, pre


def backward(params, acts, pre, dout):
    """Gradients of every (w, b) given d loss / d output."""
    grads = [None] * len(params)
    d = dout
    for li in range(len(params) - 1, -1, -1):
        if li < len(params) - 1:
            d = d * (pre[li] > 0)
        dw, db = conv3x3_grad_weight(acts[li], d)
        grads[li] = (dw, db)
        if li > 0:
            d = conv3x3_grad_input(d, params[li][0])
    return grads


def l1_loss(out, target, scale):
    """mean over pixels of sum_c scale_c |out_c - target_c|, and its gradient."""
    diff = out - target
    n = out.shape[0] * out.shape[1]
    loss = float((np.abs(diff) * scale).sum() / n)
    return loss, np.sign(diff) * scale / n
