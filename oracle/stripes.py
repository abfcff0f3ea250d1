"""Stripe-decomposed Algorithm 1 on the oracle: the multi-GPU scheme for one pair,
verified on CPU (test infrastructure only, like the rest of ``oracle/``).

The expansions of one group are independent (Lemma 3), so a pair can be split
into horizontal stripes, one per rank, with the images replicated read-only:

* stripe boundaries are multiples of every level's cell size, so a centre cell
  never straddles two stripes; rank d owns the cells whose centre cell lies in
  its stripe [top_d, bot_d) and runs their alpha_ij-expansions;
* a region reaches one cell beyond its centre cell, so rank d writes rows
  [top_d - s, bot_d + s) and reads rows [top_d - s - 1, bot_d + s + 1) (the
  pairwise terms need a 1-pixel ring);
* after every (level, group), rank d sends each neighbour the labels and cached
  costs of the pixels it changed in the rows that neighbour can ever read, and
  applies what it receives.  With stripes at least 2 s_max + 2 rows high that
  reaches everything: a write can never land in the read range of a rank two
  stripes away.

Every rank then sees, before each expansion, exactly the labels the
single-domain run sees, and the random draws are keyed by (seed, iteration,
level, cell, proposal), so the result is the single-domain result bit for bit.
"""
from __future__ import annotations

import numpy as np


def stripe_bounds(H, world, cells):
    """Row ranges of `world` stripes whose inner boundaries are multiples of the
    least common multiple of the cell sizes; raises if the stripes would be lower
    than 2 * max(cells) + 2 rows."""
    unit = int(np.lcm.reduce(np.asarray(cells, dtype=np.int64)))
    n_units = -(-H // unit)
    if n_units < world:
        raise ValueError(f"{H} rows give {n_units} boundary units of {unit} rows for {world} stripes")
    cuts = [round(k * n_units / world) * unit for k in range(world)] + [H]
    bounds = [(cuts[k], min(H, cuts[k + 1])) for k in range(world)]
    smax = max(cells)
    for t, b in bounds:
        if b - t < 2 * smax + 2 and world > 1:
            raise ValueError(f"stripe [{t}, {b}) is lower than 2 * {smax} + 2 rows")
    return bounds


def owned_cells(H, W, s, group, top, bot):
    """Cells (i, j) of `group` at cell size s whose centre cell starts in [top, bot)."""
    import oracle
    return [(i, j) for i, j in oracle.group_cells(H, W, s, group) if top <= j * s < bot]


def run_stripes(rank, world, left, right, params, n_iters, send_recv):
    """Algorithm 1 for n_iters outer iterations on stripe `rank` of `world`.

    send_recv(peer, array) sends `array` to rank `peer` and returns the array that
    peer sent back (same shape and dtype).  Returns (labels, costs) of the rows of
    this rank's stripe and the stripe's row range."""
    import oracle
    o = oracle.Oracle(left, right, **params)
    o.init_state()
    H, W = o.H, o.W
    p = o.p
    nl = p["n_levels"]
    cells = list(p["cell"])[:nl]
    smax = max(cells)
    bounds = stripe_bounds(H, world, cells)
    top, bot = bounds[rank]
    for it in range(n_iters):
        for level in range(nl):
            s = cells[level]
            for group in range(16):
                mine = owned_cells(H, W, s, group, top, bot)
                if mine:
                    o.expand_cells(it, level, mine)
                # pixels this rank may have changed: the regions of its cells
                changed = np.zeros((H, W), bool)
                for ci, cj in mine:
                    R, _ = oracle.region_of(H, W, s, ci, cj)
                    changed[R[1]:R[1] + R[3], R[0]:R[0] + R[2]] = True
                lab, cost = o.state()
                for peer in (rank - 1, rank + 1):
                    if peer < 0 or peer >= world:
                        continue
                    ptop, pbot = bounds[peer]
                    # rows the peer can ever read
                    r0, r1 = max(0, ptop - smax - 1), min(H, pbot + smax + 1)
                    out = _pack(lab[r0:r1], cost[r0:r1], changed[r0:r1])
                    got = send_recv(peer, out)
                    # the peer's band: rows this rank can ever read
                    q0, q1 = max(0, top - smax - 1), min(H, bot + smax + 1)
                    plab, pcost, pmask = _unpack(got, q1 - q0, W)
                    blab, bcost = lab[q0:q1], cost[q0:q1]
                    blab[pmask] = plab[pmask]
                    bcost[pmask] = pcost[pmask]
                o.put_state(lab, cost)
    lab, cost = o.state()
    return lab[top:bot], cost[top:bot], (top, bot)


def _pack(lab, cost, mask):
    """One float64 array: labels (as float64, exact), costs, mask; padded to a fixed size by the caller."""
    return np.concatenate([lab.astype(np.float64).ravel(), cost.ravel(), mask.astype(np.float64).ravel()])


def _unpack(buf, rows, W):
    n = rows * W
    lab = buf[:3 * n].reshape(rows, W, 3).astype(np.float32)
    cost = buf[3 * n:4 * n].reshape(rows, W)
    mask = buf[4 * n:5 * n].reshape(rows, W) > 0.5
    return lab, cost, mask
