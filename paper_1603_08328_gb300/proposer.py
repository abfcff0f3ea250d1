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

import argparse
import os
import time

import numpy as np

from .lem import ProposalNet, Stereo

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposer_384x288.npy")

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


def load(path=WEIGHTS, seed=0) -> ProposalNet:
    """A network with the weights stored at `path` (flat float32, lem_cnn_get_params order)."""
    net = ProposalNet(seed=seed)
    net.set_params(np.load(path))
    return net


def _render(args):
    from synth import workload_pair
    name, seed = args
    p = workload_pair(name, seed)
    return p["left"], p["right"]


def render_scenes(name, seeds, processes=0):
    """Synthetic pairs rendered in worker processes (spawned, so safe after CUDA use)."""
    import multiprocessing as mp
    processes = processes or min(16, os.cpu_count() or 1)
    if processes <= 1:
        return [_render((name, s)) for s in seeds]
    with mp.get_context("spawn").Pool(processes) as pool:
        return pool.map(_render, [(name, s) for s in seeds], chunksize=8)


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the plane-proposal network on synthetic scenes")
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--first-seed", type=int, default=10000)
    ap.add_argument("--chunk", type=int, default=50, help="pairs per batch handle")
    ap.add_argument("--iters", type=int, default=10, help="iterations of the plain method for the targets")
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args(argv)
    import torch
    from synth.scenes import WORKLOADS
    name = "train_384x288"
    dmax = WORKLOADS[name]["disp_max"]
    t0 = time.time()
    scenes = render_scenes(name, range(args.first_seed, args.first_seed + args.scenes))
    print(f"rendered {len(scenes)} scenes in {time.time() - t0:.1f} s", flush=True)
    t0 = time.time()
    xs, ts = [], []
    for c in range(0, len(scenes), args.chunk):
        pairs = [dict(left=l, right=r) for l, r in scenes[c:c + args.chunk]]
        x, t = make_dataset(pairs, n_in=(1, 2, 3), n_out=args.iters, disp_max=dmax, seed=c + 1)
        xs.append(x)
        ts.append(t)
    x, t = torch.cat(xs), torch.cat(ts)
    print(f"dataset {tuple(x.shape)} in {time.time() - t0:.1f} s", flush=True)
    net = ProposalNet(seed=1)
    t0 = time.time()
    losses = train(net, x, t, steps=args.steps, batch=args.batch, lr=args.lr, log_every=max(1, args.steps // 10))
    torch.cuda.synchronize()
    print(f"trained {args.steps} steps in {time.time() - t0:.1f} s: loss {np.mean(losses[:100]):.4f} -> "
          f"{np.mean(losses[-100:]):.4f}", flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, net.get_params())
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
