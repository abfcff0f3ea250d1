"""FP64 reference of the plane-proposal network (test infrastructure only).

The network maps the stereo pair and the current label map, at quarter
resolution, to per-pixel plane proposals: 6 layers of 3x3 convolutions (zero
padding, stride 1), 32 channels, ReLU after all but the last, input channels
(left RGB, right RGB, disparity), output (d, a, b).  Only the tests use this
module; it shares no code with the CUDA kernels.

Layouts: activations are (H, W, C); weights of a layer are (3, 3, Cin, Cout)
(kernel row, kernel column, input channel, output channel); y = x * w + bias
with y[v, u, o] = sum_{i,j,c} x[v + i - 1, u + j - 1, c] w[i, j, c, o].

Parity pins: tests/test_oracle_cnn.py (finite differences, scipy correlation, closed
forms of the Adam update).
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


def round_bf16(x):
    """Round to the nearest bfloat16 value (8 significant bits, ties to even), returned as
    float64.  bfloat16 is the upper half of an IEEE binary32: the value is first rounded to
    binary32, then the low 16 bits of its encoding are rounded away."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep = u >> 16
    rest = u & 0xFFFF
    up = (rest > 0x8000) | ((rest == 0x8000) & ((keep & 1) == 1))
    r = ((keep + up.astype(np.uint64)) << 16).astype(np.uint32)
    nan = np.isnan(f)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _store(x, store):
    return round_bf16(x) if store == "bf16" else x


def forward(params, x, store=None):
    """params: list of (w, b); returns the output and the per-layer inputs/pre-activations.

    store="bf16" models a kernel that keeps the weights and every layer input in bfloat16
    (the biases, pre-activations and output stay exact): those operands are rounded with
    round_bf16 where they are stored, the arithmetic stays FP64."""
    h = _store(x, store)
    acts, pre = [h], []
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, _store(w, store), b)
        pre.append(z)
        h = _store(np.maximum(z, 0.0), store) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts, pre


def backward(params, acts, pre, dout, store=None):
    """Gradients of every (w, b) given d loss / d output.  store="bf16": the gradients
    with respect to the pre-activations are kept in bfloat16 (rounded where stored) and
    the weights are the rounded ones, as in forward."""
    grads = [None] * len(params)
    d = _store(dout, store)
    for li in range(len(params) - 1, -1, -1):
        if li < len(params) - 1:
            d = _store(d * (pre[li] > 0), store)
        dw, db = conv3x3_grad_weight(acts[li], d)
        grads[li] = (dw, db)
        if li > 0:
            d = conv3x3_grad_input(d, _store(params[li][0], store))
    return grads


def l1_loss(out, target, scale):
    """mean over pixels of sum_c scale_c |out_c - target_c|, and its gradient."""
    diff = out - target
    n = out.shape[0] * out.shape[1]
    loss = float((np.abs(diff) * scale).sum() / n)
    return loss, np.sign(diff) * scale / n


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: a method for stochastic optimization",
    ICLR 2015) of the flat parameters w with gradient g, first and second moments m, v
    and 1-based step count `step`: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    w <- w - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
    Returns (w, m, v); the inputs are not changed."""
    w, g = np.asarray(w, np.float64), np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def quarter_features(left, right, lab, dmax):
    """Network input at quarter resolution: 4x4 block means (blocks clipped at the
    image border) of the left and right RGB / 255 and of the label disparity
    d_p = a u + b v + c, divided by dmax.  left/right (H, W, 3), lab (H, W, 3)."""
    H, W = lab.shape[:2]
    v, u = np.mgrid[0:H, 0:W]
    d = lab[..., 0].astype(np.float64) * u + lab[..., 1].astype(np.float64) * v + lab[..., 2]
    chans = np.concatenate([np.asarray(left, np.float64) / 255.0, np.asarray(right, np.float64) / 255.0,
                            (d / dmax)[..., None]], axis=-1)
    return _block_means(chans)


def quarter_targets(lab, dmax):
    """Training target: 4x4 block means of (d_p / dmax, a_p, b_p), the mean slopes
    clamped to [-1, 1]."""
    H, W = lab.shape[:2]
    v, u = np.mgrid[0:H, 0:W]
    lab = lab.astype(np.float64)
    d = lab[..., 0] * u + lab[..., 1] * v + lab[..., 2]
    t = _block_means(np.stack([d / dmax, lab[..., 0], lab[..., 1]], axis=-1))
    t[..., 1:] = np.clip(t[..., 1:], -1.0, 1.0)
    return t


def _block_means(x):
    H, W, C = x.shape
    H4, W4 = (H + 3) // 4, (W + 3) // 4
    out = np.zeros((H4, W4, C))
    for V in range(H4):
        for U in range(W4):
            out[V, U] = x[4 * V:4 * V + 4, 4 * U:4 * U + 4].reshape(-1, C).mean(axis=0)
    return out


def upsample_planes(y, H, W, dmax):
    """Plane label per full-resolution pixel from the quarter-resolution (d/dmax, a, b):
    bilinear interpolation at the pixel's position in the quarter grid, whose cell U
    covers pixels 4U .. 4U+3 with centre 4U + 1.5 (positions clamped to the grid), then
    c = d - a u - b v."""
    H4, W4 = y.shape[:2]
    out = np.zeros((H, W, 3))
    for vv in range(H):
        fv = min(max((vv - 1.5) / 4.0, 0.0), H4 - 1.0)
        v0 = int(fv); v1 = min(v0 + 1, H4 - 1); tv = fv - v0
        for uu in range(W):
            fu = min(max((uu - 1.5) / 4.0, 0.0), W4 - 1.0)
            u0 = int(fu); u1 = min(u0 + 1, W4 - 1); tu = fu - u0
            r = ((1 - tv) * ((1 - tu) * y[v0, u0] + tu * y[v0, u1])
                 + tv * ((1 - tu) * y[v1, u0] + tu * y[v1, u1]))
            d, a, b = r[0] * dmax, r[1], r[2]
            out[vv, uu] = (a, b, d - a * uu - b * vv)
    return out
