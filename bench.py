"""Benchmark: pixel-label cost evaluations per second of local-expansion-move stereo.

One step = one outer iteration of Algorithm 1 (3 grid levels x 16 disjoint
groups, every alpha_ij-expansion evaluated, cut and committed) on the
Middlebury-V2-shaped synthetic pair (450 x 375, disparities 0-60, cells
5/15/25 px, 41 x 41 matching windows, FP32).  Steps continue one run from the
random initialisation; warm-up steps run on a separate handle.  L2 is flushed
between timed steps; each step is timed with CUDA events on the library's
stream.

The launch configuration of every level is chosen by the library's autotuner
on the warm-up handle (it changes only the time, never a label).  A second
block measures the time to reach the plain method's energy: 10 iterations of
the plain method give E_plain; the time to E <= 1.001 E_plain is taken for the
plain method and for the method with learned proposals (when trained weights
are present), CNN inference included.

Prints one JSON line.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "middlebury_450x375"
PARAMS = dict(disp_max=60.0)          # everything else: the paper's values (lem_default_params)
METRIC = "pixel-label cost evals/s"
FP32_LANES_PER_SM = 128               # FP32 FMA lanes per SM (Blackwell)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lem", choices=["lem", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-jobs", type=int, default=2)
    ap.add_argument("--no-tune", action="store_true", help="default launch configuration")
    ap.add_argument("--launch-config", default=None,
                    help="fixed per-level configuration 'threads/gr_interval/strip_rows', each three "
                         "comma-separated values (e.g. 256,512,512/16,16,16/8,32,16); skips the autotuner")
    ap.add_argument("--no-time-to-energy", action="store_true")
    ap.add_argument("--no-proposer", action="store_true", help="skip the proposal-network timing")
    ap.add_argument("--no-bf", action="store_true", help="skip the LE-BF variant timing")
    ap.add_argument("--no-v3", action="store_true", help="skip the V3-settings timing (1500 x 1000)")
    ap.add_argument("--no-large", action="store_true", help="skip the 1500 x 1000 FP16 batched timing")
    ap.add_argument("--mode", default="step", choices=["step", "proposer", "batch8", "v3", "lebf", "large"],
                    help="proposer: time only the proposal network; batch8: the uneven batch of 8 pairs; "
                         "v3: only the V3-settings block; lebf: only the LE-BF block (one JSON line each)")
    ap.add_argument("--batch-iters", type=int, default=10, help="outer iterations per pair in --mode batch8")
    return ap.parse_args()


# --- distributed plumbing (replicas: every rank solves its own pair) -------------

def dist_init(n):
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, world, dist


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# --- clocks during the timed region ---------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# --- algorithmic work ------------------------------------------------------------

def region_geometry(H, W, s):
    """(x0, y0, w, h) of every expansion region at cell size s, by group."""
    nx, ny = -(-W // s), -(-H // s)
    groups = {g: [] for g in range(16)}
    for j in range(ny):
        for i in range(nx):
            x0, x1 = max(0, (i - 1) * s), min(W, (i + 2) * s)
            y0, y1 = max(0, (j - 1) * s), min(H, (j + 2) * s)
            groups[4 * (j % 4) + (i % 4)].append((x0, y0, x1 - x0, y1 - y0))
    return groups


def algorithmic_flops(H, W, r, x0, y0, w, h):
    """FP32 operations the data term of one candidate on region R needs: about 30 per
    raw cost over M, 44 per regression window over R grown by r' (4 box means and the
    3x3 solve) and 24 per output pixel (4 box means and the output)."""
    mw = min(W, x0 + w + 2 * r) - max(0, x0 - 2 * r)
    mh = min(H, y0 + h + 2 * r) - max(0, y0 - 2 * r)
    kw = min(W, x0 + w + r) - max(0, x0 - r)
    kh = min(H, y0 + h + r) - max(0, y0 - r)
    return 30 * mw * mh + 44 * kw * kh + 24 * w * h


def launches_and_work(H, W, p):
    r = p["gf_radius"]
    out = []
    for l in range(p["n_levels"]):
        s = p["cell"][l]
        nprop = p["k_prop"][l] + p["k_rand"][l]
        groups = region_geometry(H, W, s)
        for g in range(16):
            regs = groups[g]
            if not regs:
                continue
            evals = sum(w * h for (_, _, w, h) in regs) * nprop
            flops = sum(algorithmic_flops(H, W, r, *R) for R in regs) * nprop
            out.append(dict(level=l, group=g, evals=evals, flops=flops, regions=len(regs)))
    return out


def kernel_source_sha():
    """SHA-256 of the expansion kernel's sources: lem_kernels.cu followed by the internal
    header it includes."""
    h = hashlib.sha256()
    for name in ("lem_kernels.cu", "lem_internal.h"):
        with open(os.path.join(ROOT, "paper_1603_08328_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_from_profile(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha256") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


# --- CPU oracle ------------------------------------------------------------------

def cpu_oracle_baseline(pair, p, seed):
    """The oracle, as it stands, on the host cores: one full outer iteration (iteration
    0 from the random initialisation) of the same workload."""
    import oracle
    o = oracle.Oracle(pair["left"], pair["right"], seed=seed, **PARAMS)
    o.init_state()
    t = time.perf_counter()
    _, evals = o.iterate(0)
    dt = time.perf_counter() - t
    # the same oracle on one host core, on a smaller sample: the first two groups of the
    # finest level of iteration 1
    o1 = oracle.Oracle(pair["left"], pair["right"], seed=seed, n_threads=1, **PARAMS)
    o1.put_state(*o.state())
    t1 = time.perf_counter()
    ev1 = sum(o1.expand_group(1, 0, grp)[1] for grp in (0, 1))
    dt1 = time.perf_counter() - t1
    return {"value": evals / dt, "unit": METRIC, "cores": oracle.openmp_threads(), "kind": "oracle",
            "sample": f"outer iteration 0 of {WORKLOAD} (all 48 level-group launches, {evals} evals), "
                      f"{dt:.2f} s",
            "one_core": {"value": ev1 / dt1, "unit": METRIC, "cores": 1,
                         "sample": f"groups 0 and 1 of level 0, iteration 1 ({ev1} evals), {dt1:.2f} s"}}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores, one (level, group)
    expansion per step, cycling through the 48 of an outer iteration."""
    rank, world, dist = dist_init(args.gpus)
    if rank != 0:
        return
    import oracle
    from synth import workload_pair
    pair = workload_pair(WORKLOAD, args.seed)
    o = oracle.Oracle(pair["left"], pair["right"], seed=args.seed + 1, **PARAMS)
    o.init_state()
    nl = len(oracle.PAPER_DEFAULTS["cell"])
    seq = [(it, l, g) for it in range(1000) for l in range(nl) for g in range(16)]
    k = 0
    for _ in range(args.warmup):
        o.expand_group(*seq[k])
        k += 1
    evals = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, e = o.expand_group(*seq[k])
        evals += e
        k += 1
    dt = time.perf_counter() - t0
    v = evals / dt
    cores = oracle.openmp_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "height": 375, "width": 450, "disp_max": 60, "cells": [5, 15, 25],
                       "window": 41, "step": "one (level, group) expansion of the CPU oracle"},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} (level, group) expansions of outer iteration 0.."},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- GPU -------------------------------------------------------------------------

def conv_flops_per_pixel():
    """Algorithmic flops of one forward pass per quarter-resolution pixel: 2 * 9 * Cin * Cout
    summed over the layers, real channel counts (7 -> 32 -> ... -> 32 -> 3)."""
    layers = [(7, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 3)]
    return 2 * 9 * sum(ci * co for ci, co in layers)


def proposer_timing(lem, stream, reps=20):
    """Proposal network: forward pass on the quarter-resolution grid of a 1500 x 1000 image
    (375 x 250 x 7) and one training step (forward, both gradients and Adam) on 16 images of
    96 x 72, each timed with CUDA events (median of `reps`), as algorithmic TFLOP/s (the
    backward pass counted as twice the forward) against the measured dense BF16 peak."""
    import torch
    net = lem.ProposalNet(seed=0, stream=stream)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(250, 375, 7, device="cuda", generator=g)
    xt = torch.rand(16, 72, 96, 7, device="cuda", generator=g)
    tt = torch.rand(16, 72, 96, 3, device="cuda", generator=g)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return sorted(ts)[len(ts) // 2]

    t_fwd = timed(lambda: net.forward(x))
    t_train = timed(lambda: net.train_step(xt, tt, 1e-4))
    fpp = conv_flops_per_pixel()
    f_fwd = fpp * 250 * 375
    f_train = 3 * fpp * 16 * 72 * 96
    peak = None
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        peak_note = "of measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, ValueError, KeyError):
        peak, peak_note = 1900.0, "of fallback (1.9 PFLOP/s bf16)"
    net.close()
    fwd_tf = f_fwd / t_fwd / 1e12
    return {"forward_1500x1000_ms": 1e3 * t_fwd, "forward_tflops": fwd_tf,
            "train_step_16x96x72_ms": 1e3 * t_train, "train_tflops": f_train / t_train / 1e12,
            "flops_per_quarter_pixel": fpp, "peak_tflops": peak, "forward_frac": fwd_tf / peak,
            "peak_note": peak_note,
            "note": "BF16 implicit-GEMM convolutions: forward and input gradient on tcgen05.mma (kind::f16, TMEM accumulator), weight gradient on mma.sync m16n8k16; FP32 accumulation"}


def run_proposer_mode(args):
    """--mode proposer: only the proposal-network timing, one JSON line."""
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    __graft_entry__.build()
    from paper_1603_08328_gb300 import lem
    out = proposer_timing(lem, torch.cuda.current_stream())
    print(json.dumps({"mode": "proposer", **out}), flush=True)


def run_batch8_mode(args):
    """--mode batch8: 8 pairs from 640x480 to 2900x2000 (disparity 64-800), BF16 images,
    batched 4-candidate visits, learned proposals (k_cnn = 1 at the finest level) when
    trained weights exist, autotuned, all on one stream of one GPU.  Two runs:
      * one batch handle for all 8 pairs (one launch per (level, group) over every
        pair): aggregate evals/s;
      * one handle per pair, the pairs served one after another: per-pair latency
        (host images in, n iterations, host disparity out) p50 / p99 and aggregate.
    Prints one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    __graft_entry__.build()
    from paper_1603_08328_gb300 import lem, proposer
    from synth import BATCH8, render_batch8
    stream = torch.cuda.current_stream()
    pairs = render_batch8(args.seed)
    ranges = [(0.0, c["disp_max"]) for c in BATCH8]
    net = proposer.load() if os.path.exists(proposer.WEIGHTS) else None
    kw = dict(store_dtype=lem.LEM_STORE_BF16, candidates_per_visit=4, seed=5)
    if net is not None:
        kw["k_cnn"] = (1, 0, 0)
    n_it = args.batch_iters

    def iterate(g):
        if net is not None:
            g.cnn_propose(net)
        g.check(lem.lem_expand_iteration(g.h, 1, None))

    # tune on the largest pair's own handle (one warm-up iteration first)
    t0h = lem.Stereo(pairs[-1]["left"], pairs[-1]["right"], stream=stream, disp_max=ranges[-1][1], **kw)
    iterate(t0h)
    t = t0h.autotune(repeats=1)
    t0h.close()
    kw.update(level_threads=list(t.threads), level_gr_interval=list(t.gr_interval), level_strip_rows=list(t.strip_rows))

    # batched: one handle over all pairs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = lem.Stereo([p["left"] for p in pairs], [p["right"] for p in pairs], stream=stream, disp_ranges=ranges, **kw)
    evals_it = g.evals_per_iteration()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_it):
        iterate(g)
    b.record(stream)
    b.synchronize()
    gpu_s = a.elapsed_time(b) / 1e3
    disp = g.labels("all")[1].cpu().numpy()
    batch_job_s = time.perf_counter() - t0
    st = g.iterate(0)
    assert st.maxflow_limit == 0
    g.close()

    # served one by one: per-pair latency, host images in and host disparity out
    lat, evals_total = [], 0
    for p, rg in zip(pairs, ranges):
        H, W = p["left"].shape[:2]
        hd = torch.empty((H, W), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h1 = lem.Stereo(p["left"], p["right"], stream=stream, disp_max=rg[1], **kw)
        for _ in range(n_it):
            iterate(h1)
        lem._check(lem.lem_get_labels(h1.h, None, lem.C.c_void_p(hd.data_ptr()), None, 0), h1.h)
        lat.append(time.perf_counter() - t1)
        evals_total += h1.evals_per_iteration() * n_it
        h1.close()
    lat_ms = np.array(lat) * 1e3
    sizes = [f"{c['width']}x{c['height']}/{int(c['disp_max'])}" for c in BATCH8]
    out = {"mode": "batch8", "metric": METRIC, "unit": METRIC, "iterations": n_it,
           "pairs": sizes, "pixels": int(sum(c["width"] * c["height"] for c in BATCH8)),
           "config": {"store": "bf16", "candidates_per_visit": 4, "learned_proposals": net is not None,
                      "launch_config": {k: kw[k] for k in ("level_threads", "level_gr_interval", "level_strip_rows")}},
           "batched": {"value": evals_it * n_it / gpu_s, "gpu_ms": 1e3 * gpu_s, "job_ms": 1e3 * batch_job_s,
                       "evals": evals_it * n_it},
           "per_pair": {"value": evals_total / sum(lat), "latency_ms": [round(x, 2) for x in lat_ms],
                        "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99))},
           "disparity_finite": bool(np.isfinite(disp).all())}
    print(json.dumps(out), flush=True)


def bf_flops(H, W, r, x0, y0, w, h):
    """FP32 operations of the LE-BF data term of one candidate on region R: about 30 per
    raw cost over M (R grown by the window radius 2 r') and one multiply-add (2 flops) per
    window pixel of every output pixel, windows clipped to the image.  The colour weight of
    each window pixel (one exp2 on the special-function unit) is not counted."""
    import numpy as np
    R = 2 * r
    mw = min(W, x0 + w + R) - max(0, x0 - R)
    mh = min(H, y0 + h + R) - max(0, y0 - R)
    xs = np.arange(x0, x0 + w)
    ys = np.arange(y0, y0 + h)
    cx = np.minimum(W - 1, xs + R) - np.maximum(0, xs - R) + 1
    cy = np.minimum(H - 1, ys + R) - np.maximum(0, ys - R) + 1
    return 30 * mw * mh + 2 * int(cx.sum()) * int(cy.sum())


def bf_timing(lem, pair, stream, seed, flush, steps=3):
    """The LE-BF variant (Sec. 4: bilateral weights over the 41 x 41 window, lambda = 20)
    on the same pair: outer iterations 1 .. steps timed with CUDA events (L2 flushed
    before each), evals/s, and the data term's algorithmic FP32 rate against the FP32
    peak."""
    import torch
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, data_term=lem.LEM_DATA_BF,
                   lam=20.0, **PARAMS)
    H, W = pair["left"].shape[:2]
    g.iterate(1, stats=False)
    ts = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.check(lem.lem_expand_iteration(g.h, 1, None))
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    st = g.iterate(0)
    evals = g.evals_per_iteration()
    r = g.params.gf_radius
    flops = 0
    for l in range(g.params.n_levels):
        s = g.params.cell[l]
        nprop = g.params.k_prop[l] + g.params.k_rand[l]
        for regs in region_geometry(H, W, s).values():
            flops += nprop * sum(bf_flops(H, W, r, *R) for R in regs)
    g.close()
    t = sum(ts) / len(ts)
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    return {"ms_per_iteration": 1e3 * t, "evals_per_s": evals / t, "data_term_tflops": flops / t / 1e12,
            "frac": flops / t / 1e12 / peak, "peak_tflops": peak, "maxflow_limit": st.maxflow_limit,
            "config": "data_term = LE-BF, lambda = 20, gamma_bf = 10, default launch configuration, "
                      f"iterations 2-{steps + 1}, L2 flushed between iterations",
            "note": "whole-iteration time (cuts included); flops count only the data term"}


def large_timing(lem, stream, seed, flush, steps=3):
    """The 1500 x 1000 pair (disparity 0-400) in the production configuration: FP16 image
    storage, batched 4-candidate visits, autotuned launch configuration, outer iterations
    replayed as a CUDA graph.  Iterations 2 .. steps + 1 timed with CUDA events (L2 flushed
    before each)."""
    import torch
    from synth import workload_pair
    pair = workload_pair("large_1500x1000", 0)
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, disp_max=400.0,
                   store_dtype=lem.LEM_STORE_F16, candidates_per_visit=4)
    g.iterate(1, stats=False)
    t = g.autotune(repeats=1)
    g.iterate(1, stats=False)           # first iteration after tuning: graph capture
    ts = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.check(lem.lem_expand_iteration(g.h, 1, None))
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    st = g.iterate(0)
    evals = g.evals_per_iteration()
    g.close()
    ms = 1e3 * sum(ts) / len(ts)
    return {"workload": "large_1500x1000 (disparity 0-400), FP16 images, 4-candidate visits, autotuned, CUDA graph",
            "ms_per_iteration": ms, "evals_per_iteration": evals, "evals_per_s": evals / (ms / 1e3),
            "maxflow_limit": st.maxflow_limit,
            "launch_config": {"threads": list(t.threads), "gr_interval": list(t.gr_interval),
                              "strip_rows": list(t.strip_rows)},
            "note": f"iterations 3-{steps + 2} after one plain and one tuned iteration, L2 flushed between"}


def v3_timing(lem, stream, seed, flush):
    """The paper's Middlebury V3 settings (Sec. 4: cells of 1, 3 and 9 % of the width,
    lambda = 0.5, one RANSAC proposal per visit) on the 1500 x 1000 pair (disparity
    0-400, FP32): cells 15 / 45 / 135 px, so levels 1 and 2 (135x135 and 405x405-node
    regions) run on the multi-CTA path.  Outer iteration 1 is timed launch by launch with
    CUDA events (L2 flushed before each launch); per level: time, evals/s, cut rounds."""
    import torch
    from synth import workload_pair
    pair = workload_pair("large_1500x1000", 0)
    H, W = pair["left"].shape[:2]
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, disp_max=400.0, v3_width=W)
    g.iterate(1, stats=False)
    p = g.params
    levels = {}
    total = 0.0
    e_before = g.energy()[0]
    for l in range(p.n_levels):
        s = p.cell[l]
        nprop = p.k_prop[l] + p.k_rand[l] + p.k_rans[l]
        groups = region_geometry(H, W, s)
        d = {"cell": s, "region_nodes": min(W, 3 * s) * min(H, 3 * s), "ms": 0.0, "evals": 0, "cuts": 0,
             "path": "multi-CTA" if min(W, 3 * s) * min(H, 3 * s) > 5625 else "CTA"}
        st0 = g.iterate(0)
        for grp in range(16):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.check(lem.lem_expand_group(g.h, 1, l, grp, None))
            b.record(stream)
            b.synchronize()
            d["ms"] += a.elapsed_time(b)
            d["evals"] += sum(w * h for (_, _, w, h) in groups[grp]) * nprop
            d["cuts"] += len(groups[grp]) * nprop
        st = g.iterate(0)
        d["rounds_per_cut"] = st.pr_rounds / max(1, d["cuts"])
        d["relabels_per_cut"] = st.pr_global_relabels / max(1, d["cuts"])
        d["bfs_levels_per_relabel"] = st.pr_bfs_levels / max(1, st.pr_global_relabels)
        d["maxflow_limit"] = st.maxflow_limit
        d["evals_per_s"] = d["evals"] / (d["ms"] / 1e3)
        total += d["ms"]
        levels[str(l)] = d
    e_after = g.energy()[0]
    evals = g.evals_per_iteration()
    g.close()
    return {"workload": "large_1500x1000 (disparity 0-400, FP32 images), V3 settings: cells 1/3/9 % of the width, "
                        "lambda 0.5, K_RANS 1", "ms_per_iteration": total, "evals_per_s": evals / (total / 1e3),
            "evals_per_iteration": evals, "energy": {"before": e_before, "after": e_after}, "levels": levels,
            "note": "iteration 1, one lem_expand_group call per (level, group), L2 flushed before each"}


def time_to_energy(lem, pair, params, stream, seed, n_plain=10, max_iters=10):
    """Time (CUDA events around each outer iteration, learned proposals' inference
    included) to reach E <= 1.001 E_plain, E_plain the energy after n_plain iterations of
    the plain method, for the plain method and for the learned proposer (k_cnn = 1 at the
    finest level) when its trained weights are present."""
    import torch
    from paper_1603_08328_gb300 import proposer

    def run(g, net, n):
        curve, t = [], 0.0
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if net is not None:
                g.cnn_propose(net)
            g.check(lem.lem_expand_iteration(g.h, 1, None))
            b.record(stream)
            b.synchronize()
            t += a.elapsed_time(b)
            curve.append((g.energy()[0], t))
        return curve

    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, **params)
    plain = run(g, None, n_plain)
    g.close()
    target = 1.001 * plain[-1][0]

    def first(curve):
        for k, (e, t) in enumerate(curve):
            if e <= target:
                return k + 1, t
        return None, None

    pi, pt = first(plain)
    out = {"target_energy": target, "plain_energy": plain[-1][0], "plain_iters": pi, "plain_ms": pt,
           "plain_curve": [[round(e, 1), round(t, 2)] for e, t in plain]}
    if not os.path.exists(proposer.WEIGHTS):
        out["learned"] = "no trained weights"
        return out
    net = proposer.load()
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, k_cnn=(1, 0, 0), **params)
    curve = run(g, net, max_iters)
    g.close()
    li, lt = first(curve)
    out.update({"learned_iters": li, "learned_ms": lt, "learned_energy": curve[-1][0],
                "learned_curve": [[round(e, 1), round(t, 2)] for e, t in curve],
                "speedup": (pt / lt) if (pt and lt) else None,
                "learned_config": "k_cnn = (1, 0, 0), proposal map refreshed before every iteration"})
    net.close()
    return out

def _block(fn, *a, **kw):
    """One extra measurement; an exception becomes {"error": ...} in the JSON line."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"}


def run_lem(args):
    import numpy as np
    import torch

    import __graft_entry__
    rank, world, dist = dist_init(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    dev = torch.cuda.current_device()
    if rank == 0 or dist is None:
        __graft_entry__.build()
    barrier(dist)
    from paper_1603_08328_gb300 import lem
    from synth import workload_pair

    pair = workload_pair(WORKLOAD, args.seed + rank)
    stream = torch.cuda.current_stream()
    H, W = pair["left"].shape[:2]

    # warm-up: a separate handle, W outer iterations, then the autotuner on its state
    warm = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=1000 + rank, **PARAMS)
    warm.iterate(max(1, args.warmup), stats=False)
    tuned = {}
    tuning = None
    if args.launch_config:
        t3 = [[int(x) for x in part.split(",")] for part in args.launch_config.split("/")]
        tuned = dict(level_threads=t3[0], level_gr_interval=t3[1], level_strip_rows=t3[2])
        tuning = dict(tuned, source="--launch-config")
    elif not args.no_tune:
        t = warm.autotune(repeats=2)
        tuned = dict(level_threads=list(t.threads), level_gr_interval=list(t.gr_interval),
                     level_strip_rows=list(t.strip_rows))
        tuning = dict(tuned, ms=[round(x, 4) for x in t.ms], ms_default=[round(x, 4) for x in t.ms_default],
                      configs_tried=t.configs_tried)
    torch.cuda.synchronize()
    warm.close()
    params = dict(PARAMS, **tuned)

    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=1 + rank, **params)
    p = dict(gf_radius=g.params.gf_radius, n_levels=g.params.n_levels, cell=list(g.params.cell),
             k_prop=list(g.params.k_prop), k_rand=list(g.params.k_rand))
    work = launches_and_work(H, W, p)
    evals_per_step = g.evals_per_iteration()
    assert evals_per_step == sum(x["evals"] for x in work)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    e0, q0 = g.energy()
    g.iterate(0)                       # stats baseline: counters restart here
    times = []
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.check(lem.lem_expand_iteration(g.h, 1, None))
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
    torch.cuda.synchronize()
    t_total = sum(times)
    t_max = max_over_ranks(t_total, dist)
    e1, q1 = g.energy()
    st = g.iterate(0)
    assert st.maxflow_limit == 0, "a cut hit its round limit"

    # per-launch durations of the expansion kernel (one launch per lem_expand_group call),
    # on a fresh handle over one outer iteration, L2 flushed before every launch
    g2 = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=1 + rank, **params)
    per, cut = [], []
    for wk in work:
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        sts = lem.lem_stats()
        a.record(stream)
        g2.check(lem.lem_expand_group(g2.h, 0, wk["level"], wk["group"], None))
        b.record(stream)
        b.synchronize()
        per.append(a.elapsed_time(b) / 1e3)
        lem.lib().lem_expand_iteration(g2.h, 0, lem.C.byref(sts))
        cut.append((sts.pr_rounds, sts.pr_global_relabels, sts.pr_bfs_levels))
    g2.close()
    flops = sum(wk["flops"] for wk in work)
    launch_avg = sum(per) / len(per)
    achieved = flops / len(work) / launch_avg / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    by_level = {}
    for wk, t, c in zip(work, per, cut):
        d = by_level.setdefault(wk["level"], {"ms": 0.0, "evals": 0, "flops": 0, "launches": 0, "cuts": 0,
                                              "rounds": 0, "relabels": 0, "bfs_levels": 0})
        d["ms"] += 1e3 * t
        d["evals"] += wk["evals"]
        d["flops"] += wk["flops"]
        d["launches"] += 1
        lv = wk["level"]
        d["cuts"] += wk["regions"] * (p["k_prop"][lv] + p["k_rand"][lv])
        d["rounds"] += c[0]
        d["relabels"] += c[1]
        d["bfs_levels"] += c[2]

    # end to end through the C ABI: pinned host images in, disparity map out,
    # one job = create + 10 outer iterations
    n_iters_job = 10
    hl = torch.from_numpy(pair["left"]).pin_memory()
    hr = torch.from_numpy(pair["right"]).pin_memory()
    hd = torch.empty((H, W), dtype=torch.float32).pin_memory()
    e2e_t = []
    for j in range(args.e2e_jobs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prm = lem.lem_default_params(seed=7 + j, **params)
        prm.stream = stream.cuda_stream
        li = lem.lem_image(hl.data_ptr(), H, W, 3 * W, 0)
        ri = lem.lem_image(hr.data_ptr(), H, W, 3 * W, 0)
        h = lem.lem_create(li, ri, prm)
        lem._check(lem.lem_expand_iteration(h, n_iters_job, None), h)
        lem._check(lem.lem_get_labels(h, None, lem.C.c_void_p(hd.data_ptr()), None, 0), h)
        e2e_t.append(time.perf_counter() - t0)
        lem.lem_destroy(h)
    e2e_job = max_over_ranks(sum(e2e_t) / len(e2e_t), dist)
    e2e_v = world * n_iters_job * evals_per_step / e2e_job

    # the extra blocks report their own failure instead of taking the headline line with
    # them; only rank 0 prints them, so only rank 0 runs them
    extra = rank == 0
    tte = None if args.no_time_to_energy or not extra else _block(time_to_energy, lem, pair, params, stream, seed=21)
    prop = None if args.no_proposer or not extra else _block(proposer_timing, lem, stream)
    lebf = None if args.no_bf or not extra else _block(bf_timing, lem, pair, stream, seed=31, flush=flush)
    v3 = None if args.no_v3 or not extra else _block(v3_timing, lem, stream, seed=41, flush=flush)
    large = None if args.no_large or not extra else _block(large_timing, lem, stream, seed=51, flush=flush)

    if rank != 0:
        return
    value = world * evals_per_step * args.steps / t_max
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "height": H, "width": W, "disp_max": 60, "cells": p["cell"],
                   "window": 4 * p["gf_radius"] + 1, "step": "one outer iteration (48 level-group launches)",
                   "schedule": "sequential proposals (Algorithm 2)", "l2": "flushed between timed steps",
                   "launch_config": tuning or "default",
                   "parallelism": f"replicas x{world}", "evals_per_step": evals_per_step},
        "e2e": {"value": e2e_v, "unit": METRIC, "h2d_bytes_per_step": 2 * H * W * 3, "d2h_bytes_per_step": H * W * 4,
                "step": f"one job: host images -> lem_create -> {n_iters_job} iterations -> host disparity",
                "jobs": args.e2e_jobs, "ms_per_job": 1e3 * e2e_job},
        # the first step launches the 48 (level, group) kernels directly; later steps replay
        # them as one CUDA graph that also increments the device iteration index
        "gpu_launches": len(work) * args.steps + max(0, args.steps - 1),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic_from_profile("k_expand_group"), "kernel": "k_expand_group",
                     "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz",
                     "launch_avg_ms": 1e3 * launch_avg},
        "clocks": clk.summary(),
        "energy": {"before": e0, "after": e1},
        "time_to_energy": tte,
        "proposer": prop,
        "le_bf": lebf,
        "v3": v3,
        "large": large,
        "levels": {str(k): {"ms": round(v["ms"], 3), "launches": v["launches"],
                            "evals_per_s": v["evals"] / (v["ms"] / 1e3),
                            "tflops": v["flops"] / (v["ms"] / 1e3) / 1e12,
                            # one cut per candidate and region, one node per pixel of the region
                            "cuts_per_s": v["cuts"] / (v["ms"] / 1e3),
                            "nodes_per_cut": v["evals"] / max(1, v["cuts"]),
                            "rounds_per_cut": v["rounds"] / max(1, v["cuts"]),
                            "relabels_per_cut": v["relabels"] / max(1, v["cuts"]),
                            "bfs_levels_per_relabel": v["bfs_levels"] / max(1, v["relabels"])}
                   for k, v in by_level.items()},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = _block(cpu_oracle_baseline, pair, p, seed=1)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_block_mode(args):
    """--mode v3 / lebf / large: one of the extra blocks of the default run on its own."""
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    __graft_entry__.build()
    from paper_1603_08328_gb300 import lem
    from synth import workload_pair
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if args.mode == "v3":
        out = v3_timing(lem, stream, seed=41, flush=flush)
    elif args.mode == "large":
        out = large_timing(lem, stream, seed=51, flush=flush)
    else:
        out = bf_timing(lem, workload_pair(WORKLOAD, args.seed), stream, seed=31, flush=flush)
    print(json.dumps({"mode": args.mode, **out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode in ("v3", "lebf", "large"):
        run_block_mode(args)
    elif args.mode == "proposer":
        run_proposer_mode(args)
    elif args.mode == "batch8":
        run_batch8_mode(args)
    else:
        run_lem(args)


if __name__ == "__main__":
    main()
