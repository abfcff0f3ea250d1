"""Training and use of the learned plane proposer (an extension of the method).

The network (lem_cnn_* entry points) sees the stereo pair and the current label map at
quarter resolution and predicts, per quarter-resolution pixel, the disparity and slopes
(d, a, b) of the labels the method converges to.  Its upsampled prediction is a
proposal map: with k_cnn > 0, every region visit also tries k_cnn labels of that map
(drawn from the centre cell as propagation draws its pixel), so the expansion moves
can jump to the network's plane where the current labels are still far from it.

Training data come from the method itself (self-distillation): batch handles run
Algorithm 1 on synthetic pairs; the labels after 1 .. n_in iterations give the inputs,
the labels after n_out iterations the targets.  No CPU path: every step runs in the
CUDA library.
"""
from __future__ import annotations

import time

import numpy as np

from .lem import ProposalNet, Stereo

# Disparity is predicted as d / disp_max (order 1); the slopes are small (|a|, |b| < 1),
# so they are weighted up in the L1 loss.
LOSS_SCALE = (1.0, 4.0, 4.0)


def make_dataset(pairs, n_in=(1, 2), n_out=8, **params):
    """pairs: list of synthetic pairs (dicts with 'left', 'right').  Returns (x, t) CUDA
    tensors of shapes (len(pairs) * len(n_in), H4, W4, 7) and (..., 3)."""
    import torch
    s = Stereo([p["left"] for p in pairs], [p["right"] for p in pairs], **params)
    xs, done = [], 0
    for k in sorted(n_in):
        s.iterate(k - done, stats=False)
        done = k
        xs.append(torch.stack([s.cnn_features(b) for b in range(len(pairs))]))
    s.iterate(n_out - done, stats=False)
    t = torch.stack([s.cnn_targets(b) for b in range(len(pairs))])
    x = torch.cat(xs)
    t = t.repeat(len(n_in), 1, 1, 1)
    torch.cuda.synchronize()
    s.close()
    return x, t


def train(net: ProposalNet, x, t, steps=400, batch=8, lr=1e-3, seed=0, log_every=0):
    """Adam on random mini-batches of the dataset; returns the loss of every step."""
    import torch
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    losses = []
    for k in range(steps):
        idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device=x.device)
        # cosine decay of the rate to 10% of lr
        rate = lr * (0.1 + 0.9 * 0.5 * (1.0 + np.cos(np.pi * k / max(1, steps))))
        losses.append(net.train_step(x[idx], t[idx], float(rate), LOSS_SCALE))
        if log_every and k % log_every == 0:
            print(f"step {k}: loss {losses[-1]:.4f}")
    return losses


def solve(stereo: Stereo, n_iters, net: ProposalNet | None = None, first=1):
    """Algorithm 1 for n_iters outer iterations; with a network the proposal map is
    refreshed from the current labels before every iteration from `first` on (before
    that it holds the network's prediction from the initial labels).  Returns the energy
    and wall time after each iteration."""
    import torch
    out = []
    t0 = time.perf_counter()
    for it in range(n_iters):
        if net is not None and (it >= first or it == 0):
            stereo.cnn_propose(net)
        st = stereo.iterate(1)
        torch.cuda.synchronize()
        out.append((st.energy, time.perf_counter() - t0, st.evals))
    return out
