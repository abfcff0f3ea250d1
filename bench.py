"""Benchmark: pixel-label cost evaluations per second of local-expansion-move stereo.

Headline workload: the 1500 x 1000 pair (disparities 0-400, ~40 slanted and
curved segments), images stored in FP16, costs in FP32, every region of a cell
group evaluated with 4 candidate labels per visit in one launch whose
co-resident CTAs drain a work queue of the group's regions (largest first),
outer iterations replayed as CUDA graphs, launch configuration chosen by the
library's autotuner.

One step = one outer iteration of Algorithm 1 (3 grid levels x 16 disjoint
groups).  A handle runs the method's 10 outer iterations (Sec. 4 settings) and
no more: step i is iteration i mod 10 of handle i div 10, so every timed step is
an iteration the method actually runs.  Warm-up iterations and the autotuner
run on a separate handle.  L2 is flushed between timed steps; each step is timed
with CUDA events on the library's stream, and the library records events
between its launches (lem_set_kernel_timing) so the time of each kernel kind
comes from the timed steps themselves.

Beside the headline the JSON line carries:
  * e2e        : whole jobs through the C ABI (pinned host images -> lem_create ->
                 10 iterations -> host disparity);
  * roofline   : the dominant kernel's algorithmic work over its time in the timed
                 steps, against the FP32 FMA peak measured by the library's own
                 microbenchmark (lem_measure_peaks) on this GPU;
  * time_to_energy_ms / plain_ms / speedup : time to E <= 1.001 E_plain, E_plain
                 the energy of the plain method (sequential proposals, FP32 images)
                 after its 10 iterations, with learned proposals plus batched visits,
                 against the plain method itself, on the same pair and GPU;
  * cpu_baseline: the FP64 oracle on the host cores, one outer iteration of the
                 same workload (per-iteration only).
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

WORKLOAD = "large_1500x1000"
DISP_MAX = 400.0
ITERS_PER_HANDLE = 10                 # the method's outer iterations (Sec. 4)
METRIC = "pixel-label cost evals/s"


def headline_params(lem):
    """The headline configuration: the paper's settings, FP16 image storage, 4-candidate visits,
    one dataflow launch per level (the 16 groups' regions in one work queue, largest first
    within a group, each region waiting only for the overlapping regions of earlier groups)."""
    return dict(disp_max=DISP_MAX, store_dtype=lem.LEM_STORE_F16, candidates_per_visit=4, work_queue=1,
                dataflow=1)


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
                    help="fixed launch configuration instead of the autotuner's, as threads/relabel interval/"
                         "strip rows per level, e.g. 256,512,512/8,16,16/12,32,12 (for profiling captures)")
    ap.add_argument("--no-time-to-energy", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra blocks (proposer, LE-BF, V3, 450x375)")
    ap.add_argument("--mode", default="step", choices=["step", "proposer", "batch8", "v3", "lebf", "cnn_gain"],
                    help="proposer: time only the proposal network; batch8: the uneven batch of 8 pairs; "
                         "v3 / lebf: one extra block; cnn_gain: learned proposals on held-out seeds "
                         "(one JSON line each)")
    ap.add_argument("--batch-iters", type=int, default=10, help="outer iterations per pair in --mode batch8")
    ap.add_argument("--seeds", type=int, default=20, help="held-out seeds of --mode cnn_gain")
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


def iteration_work(H, W, p):
    """Per level: pixel-label evals and data-term flops of one outer iteration (every
    candidate of every region)."""
    r = p["gf_radius"]
    out = {}
    for l in range(p["n_levels"]):
        s = p["cell"][l]
        nprop = p["k_prop"][l] + p["k_rand"][l]
        evals = flops = 0
        for regs in region_geometry(H, W, s).values():
            evals += sum(w * h for (_, _, w, h) in regs) * nprop
            flops += sum(algorithmic_flops(H, W, r, *R) for R in regs) * nprop
        out[l] = dict(evals=evals, flops=flops)
    return out


def kernel_source_sha():
    """SHA-256 of the expansion kernels' sources: lem_kernels.cu followed by the internal
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


def measured_peaks(lem, stream):
    """FP32 FMA TFLOP/s and shared-memory GB/s of this GPU from the library's
    microbenchmarks, with the SM clocks sampled while they ran."""
    import torch
    dev = torch.cuda.current_device()
    with ClockSampler(dev) as clk:
        time.sleep(0.3)
        fp32, smem = lem.lem_measure_peaks(stream)
        fp32b, smemb = lem.lem_measure_peaks(stream)
        time.sleep(0.3)
    return {"fp32_tflops": max(fp32, fp32b), "smem_gbs": max(smem, smemb), "clocks": clk.summary(),
            "how": "lem_measure_peaks: FMA chains on every SM (8 CTAs x 256 threads per SM) and 16-byte "
                   "conflict-free shared loads (2 CTAs x 1024 threads per SM), best of 5 launches each"}


# --- CPU oracle ------------------------------------------------------------------

ORACLE_PARAMS = dict(disp_max=DISP_MAX, visit=4)   # the headline schedule (images are FP64 in the oracle)


def cpu_oracle_baseline(pair, seed):
    """The oracle, as it stands, on the host cores: one full outer iteration (iteration
    0 from the random initialisation) of the headline workload, per-iteration only; and
    on one host core, the first 2400 cells of group 0 of the finest level."""
    import oracle
    o = oracle.Oracle(pair["left"], pair["right"], seed=seed, **ORACLE_PARAMS)
    o.init_state()
    t = time.perf_counter()
    _, evals = o.iterate(0)
    dt = time.perf_counter() - t
    o1 = oracle.Oracle(pair["left"], pair["right"], seed=seed, n_threads=1, **ORACLE_PARAMS)
    o1.put_state(*o.state())
    H, W = pair["left"].shape[:2]
    cells = oracle.group_cells(H, W, 5, 0)[:2400]
    t1 = time.perf_counter()
    _, ev1 = o1.expand_cells(1, 0, cells)
    dt1 = time.perf_counter() - t1
    return {"value": evals / dt, "unit": METRIC, "cores": oracle.openmp_threads(), "kind": "oracle",
            "sample": f"outer iteration 0 of {WORKLOAD} (4-candidate visits, all 48 level-group steps, "
                      f"{evals} evals), {dt:.2f} s; per-iteration only",
            "one_core": {"value": ev1 / dt1, "unit": METRIC, "cores": 1,
                         "sample": f"2400 cells of group 0 of level 0, iteration 1 ({ev1} evals), {dt1:.2f} s"}}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores on the headline
    workload, one (level, group) step of the batched schedule per step, cycling
    through the 48 of an outer iteration."""
    rank, world, dist = dist_init(args.gpus)
    if rank != 0:
        return
    import oracle
    from synth import workload_pair
    pair = workload_pair(WORKLOAD, args.seed)
    H, W = pair["left"].shape[:2]
    o = oracle.Oracle(pair["left"], pair["right"], seed=args.seed + 1, **ORACLE_PARAMS)
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
            "config": {"workload": WORKLOAD, "height": H, "width": W, "disp_max": DISP_MAX, "cells": [5, 15, 25],
                       "window": 41, "candidates_per_visit": 4,
                       "step": "one (level, group) step of the FP64 CPU oracle"},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} (level, group) steps of outer iteration 0.. of {WORKLOAD}"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
            "note": "BF16 implicit-GEMM convolutions on tcgen05.mma (kind::f16, TMEM accumulators): forward, input "
                    "gradient, and weight gradient (per-CTA partials in tensor memory, added in a fixed order); "
                    "FP32 accumulation"}


def run_batch8_mode(args):
    """--mode batch8: 8 pairs from 640x480 to 2900x2000 (disparity 64-800), BF16 images,
    batched 4-candidate visits, learned proposals (k_cnn = 1 at the finest level) when
    trained weights exist, autotuned, all on one stream of one GPU.  Two runs:
      * one batch handle for all 8 pairs (one launch per (level, group) over every
        pair): aggregate evals/s;
      * one handle per pair, the pairs served one after another: per-pair latency
        (host images in, n iterations, host disparity out) p50 / p99 and aggregate.
    Both with one CTA per region and with work-queue launches (work_queue = 1, largest
    regions first); the better batched throughput is `value`.  Prints one JSON line."""
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

    def one_setting(kw):
        # batched: one handle over all pairs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = lem.Stereo([p["left"] for p in pairs], [p["right"] for p in pairs], stream=stream, disp_ranges=ranges,
                       **kw)
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
        return {"batched": {"value": evals_it * n_it / gpu_s, "gpu_ms": 1e3 * gpu_s, "job_ms": 1e3 * batch_job_s,
                            "evals": evals_it * n_it},
                "per_pair": {"value": evals_total / sum(lat), "latency_ms": [round(x, 2) for x in lat_ms],
                             "p50_ms": float(np.percentile(lat_ms, 50)),
                             "p99_ms": float(np.percentile(lat_ms, 99))},
                "disparity_finite": bool(np.isfinite(disp).all())}

    runs = {"one_cta_per_region": one_setting(dict(kw, work_queue=0)),
            "work_queue": one_setting(dict(kw, work_queue=1)),
            "dataflow": one_setting(dict(kw, work_queue=1, dataflow=1))}
    best = max(runs, key=lambda k: runs[k]["batched"]["value"])
    sizes = [f"{c['width']}x{c['height']}/{int(c['disp_max'])}" for c in BATCH8]
    out = {"mode": "batch8", "metric": METRIC, "unit": METRIC, "iterations": n_it,
           "pairs": sizes, "pixels": int(sum(c["width"] * c["height"] for c in BATCH8)),
           "config": {"store": "bf16", "candidates_per_visit": 4, "learned_proposals": net is not None,
                      "launch_config": {k: kw[k] for k in ("level_threads", "level_gr_interval", "level_strip_rows")}},
           "best": best, "value": runs[best]["batched"]["value"], **runs}
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


def bf_timing(lem, pair, stream, seed, flush, steps=3, fp32_peak=None):
    """The LE-BF variant (Sec. 4: bilateral weights over the 41 x 41 window, lambda = 20)
    on the 450 x 375 pair (disparities 0-60, sequential proposals, FP32 images): outer
    iterations 2 .. steps + 1 timed with CUDA events (L2 flushed before each), evals/s,
    and the data term's algorithmic FP32 rate against the measured FP32 peak."""
    import torch
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=seed, data_term=lem.LEM_DATA_BF,
                   lam=20.0, disp_max=60.0)
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
    peak = fp32_peak if fp32_peak else lem.lem_measure_peaks(stream)[0]
    return {"ms_per_iteration": 1e3 * t, "evals_per_s": evals / t, "data_term_tflops": flops / t / 1e12,
            "frac": flops / t / 1e12 / peak, "peak_tflops": peak, "peak_note": "of measured (lem_measure_peaks)",
            "maxflow_limit": st.maxflow_limit,
            "config": "data_term = LE-BF, lambda = 20, gamma_bf = 10, default launch configuration, "
                      f"iterations 2-{steps + 1}, L2 flushed between iterations",
            "note": "whole-iteration time (cuts included); flops count only the data term"}


def v3_timing(lem, stream, seed, flush, pair=None):
    """The paper's Middlebury V3 settings (Sec. 4: cells of 1, 3 and 9 % of the width,
    lambda = 0.5, one RANSAC proposal per visit) on the 1500 x 1000 pair (disparity
    0-400, FP32): cells 15 / 45 / 135 px, so levels 1 and 2 (135x135 and 405x405-node
    regions) run on the multi-CTA path.  Outer iteration 1 is timed launch by launch with
    CUDA events (L2 flushed before each launch); per level: time, evals/s, cut rounds."""
    import torch
    from synth import workload_pair
    if pair is None:
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


def _block(fn, *a, **kw):
    """One extra measurement; an exception becomes {"error": ...} in the JSON line."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"}


# --- GPU -------------------------------------------------------------------------

def timed_iteration(lem, g, stream, flush=None):
    """One outer iteration of handle g between CUDA events on the library's stream
    (L2 flushed first when a buffer is given): seconds."""
    import torch
    if flush is not None:
        flush.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.check(lem.lem_expand_iteration(g.h, 1, None))
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def time_to_energy(lem, pair, stream, tuned, seed=21, n_plain=ITERS_PER_HANDLE, max_iters=ITERS_PER_HANDLE):
    """Time to E <= 1.001 E_plain on one pair, E_plain the energy of the plain method (the
    paper's schedule: sequential proposals, FP32 images) after its 10 iterations, for
      * the plain method itself (autotuned after its first iteration, which is timed; the same
        dataflow launches as the others, which change no result);
      * batched visits (4 candidates, FP16 images), the headline configuration;
      * batched visits plus learned proposals (k_cnn = 1 at the finest level, the proposal
        map refreshed by the network before every iteration, inference timed).
    Times are CUDA events around each iteration (autotuning excluded)."""
    from paper_1603_08328_gb300 import proposer

    def run(g, net, n, tune=False):
        curve, t = [], 0.0
        for k in range(n):
            import torch
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
            if tune and k == 0:
                g.autotune(repeats=1)
        return curve

    base = dict(disp_max=DISP_MAX, seed=seed)
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, work_queue=1, dataflow=1, **base)
    plain = run(g, None, n_plain, tune=True)
    g.close()
    target = 1.001 * plain[-1][0]

    def first(curve):
        for k, (e, t) in enumerate(curve):
            if e <= target:
                return k + 1, t
        return None, None

    pi, pt = first(plain)
    out = {"target_energy": target, "plain_energy": plain[-1][0], "plain_iters": pi, "plain_ms": pt,
           "plain_curve": [[round(e, 1), round(t, 2)] for e, t in plain],
           "plain_config": "sequential proposals (Algorithm 2), FP32 images, dataflow launches, autotuned after "
                           "iteration 1"}
    fast = dict(base, **headline_params(lem), **tuned)
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, **fast)
    bat = run(g, None, max_iters)
    g.close()
    bi, bt = first(bat)
    out.update({"batched_iters": bi, "batched_ms": bt, "batched_curve": [[round(e, 1), round(t, 2)] for e, t in bat]})
    if not os.path.exists(proposer.WEIGHTS):
        out["learned"] = "no trained weights"
        return out
    net = proposer.load()
    g = lem.Stereo(pair["left"], pair["right"], stream=stream, k_cnn=(1, 0, 0), **fast)
    curve = run(g, net, max_iters)
    g.close()
    net.close()
    li, lt = first(curve)
    out.update({"learned_iters": li, "learned_ms": lt, "learned_energy": curve[-1][0],
                "learned_curve": [[round(e, 1), round(t, 2)] for e, t in curve],
                "speedup": (pt / lt) if (pt and lt) else None,
                "learned_config": "batched visits (4 candidates, FP16 images) + k_cnn = (1, 0, 0), proposal map "
                                  "refreshed before every iteration"})
    return out


def middlebury_timing(lem, stream, flush, steps=3):
    """The 450 x 375 Middlebury-V2-shaped pair (disparities 0-60) with the paper's
    schedule (sequential proposals, FP32 images): iterations 2 .. steps + 1, L2 flushed
    before each, kernel times from the library's events; once with the default launch
    shape and group launches, once autotuned (after iteration 1) with dataflow launches
    (the same labels)."""
    from synth import workload_pair
    pair = workload_pair("middlebury_450x375", 0)

    def one(**kw):
        g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=61, disp_max=60.0, **kw)
        g.set_kernel_timing(True)
        g.iterate(1, stats=False)
        tuned = None
        if kw:
            t = g.autotune(repeats=1)
            tuned = [list(t.threads), list(t.gr_interval), list(t.strip_rows)]
        ts, kt = [], {}
        for _ in range(steps):
            ts.append(timed_iteration(lem, g, stream, flush))
            for (l, k), (ms, n) in g.kernel_times().items():
                kt[f"{k} level {l}"] = kt.get(f"{k} level {l}", 0.0) + ms
        st = g.iterate(0)
        evals = g.evals_per_iteration()
        g.close()
        t = sum(ts) / len(ts)
        out = {"ms_per_iteration": 1e3 * t, "evals_per_s": evals / t, "maxflow_limit": st.maxflow_limit,
               "kernel_ms_per_iteration": {k: v / steps for k, v in kt.items()}}
        if tuned:
            out["launch_config"] = tuned
        return out

    return {"workload": "middlebury_450x375 (disparity 0-60), FP32 images, sequential proposals",
            "default": one(), "tuned_dataflow": one(work_queue=1, dataflow=1),
            "note": f"iterations 2-{steps + 1}, L2 flushed between; default = group launches with the default launch "
                    f"configuration, tuned_dataflow = dataflow launches autotuned after iteration 1"}


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
    params = headline_params(lem)

    # warm-up: a separate handle, W outer iterations (at most the method's 10), then the
    # autotuner on its state
    warm = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=1000 + rank, **params)
    warm.iterate(min(ITERS_PER_HANDLE, max(1, args.warmup)), stats=False)
    tuned, tuning = {}, "default"
    if args.launch_config:
        th, gr, sr = ([int(x) for x in part.split(",")] for part in args.launch_config.split("/"))
        tuned = dict(level_threads=th, level_gr_interval=gr, level_strip_rows=sr)
        tuning = dict(tuned, fixed=True)
    elif not args.no_tune:
        t = warm.autotune(repeats=1)
        tuned = dict(level_threads=list(t.threads), level_gr_interval=list(t.gr_interval),
                     level_strip_rows=list(t.strip_rows))
        tuning = dict(tuned, ms=[round(x, 4) for x in t.ms], ms_default=[round(x, 4) for x in t.ms_default],
                      configs_tried=t.configs_tried)
    torch.cuda.synchronize()
    warm.close()
    params = dict(params, **tuned)

    pinfo = None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    times, kt, launches, evals_total, graph_steps = [], {}, 0, 0, 0
    e_first = e_last = None
    g = None
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            if i % ITERS_PER_HANDLE == 0:
                # a new handle (new random initialisation) every 10 iterations: created and
                # initialised outside the timed iterations
                if g is not None:
                    e_last = g.energy()[0]
                    st = g.iterate(0)
                    assert st.maxflow_limit == 0, "a cut hit its round limit"
                    g.close()
                g = lem.Stereo(pair["left"], pair["right"], stream=stream, seed=1 + rank + 7919 * (i // 10), **params)
                g.set_kernel_timing(True)
                g.iterate(0)
                if e_first is None:
                    e_first = g.energy()[0]
                if pinfo is None:
                    pinfo = dict(gf_radius=g.params.gf_radius, n_levels=g.params.n_levels,
                                 cell=list(g.params.cell), k_prop=list(g.params.k_prop),
                                 k_rand=list(g.params.k_rand))
                torch.cuda.synchronize()
            times.append(timed_iteration(lem, g, stream, flush))
            for key, (ms, n) in g.kernel_times().items():
                d = kt.setdefault(key, [0.0, 0])
                d[0] += ms
                d[1] += n
                launches += n
            graph_steps += 1 if i % ITERS_PER_HANDLE else 0
            evals_total += g.evals_per_iteration()
    torch.cuda.synchronize()
    e_last = g.energy()[0]
    st = g.iterate(0)
    assert st.maxflow_limit == 0, "a cut hit its round limit"
    evals_per_step = g.evals_per_iteration()
    g.close()
    t_total = sum(times)
    t_max = max_over_ranks(t_total, dist)

    # per kernel kind: time and launches in the timed steps, and the levels it ran
    work = iteration_work(H, W, pinfo)
    peaks = measured_peaks(lem, stream) if rank == 0 else None
    kinds = {}
    for (l, k), (ms, n) in kt.items():
        d = kinds.setdefault(k, {"ms": 0.0, "launches": 0, "levels": []})
        d["ms"] += ms
        d["launches"] += n
        d["levels"].append(l)
    dom = max(kinds.items(), key=lambda kv: kv[1]["ms"])[0]
    roof = {"kernel": dom,
            "kernel_ms_per_step": {f"{k} level {l}": round(v[0] / args.steps, 4) for (l, k), v in sorted(kt.items())},
            "launches_per_step": {f"{k} level {l}": v[1] / args.steps for (l, k), v in sorted(kt.items())}}

    # end to end through the C ABI: pinned host images in, disparity map out,
    # one job = create + 10 outer iterations
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
        lem._check(lem.lem_expand_iteration(h, ITERS_PER_HANDLE, None), h)
        lem._check(lem.lem_get_labels(h, None, lem.C.c_void_p(hd.data_ptr()), None, 0), h)
        e2e_t.append(time.perf_counter() - t0)
        lem.lem_destroy(h)
    e2e_job = max_over_ranks(sum(e2e_t) / len(e2e_t), dist)
    e2e_v = world * ITERS_PER_HANDLE * evals_per_step / e2e_job

    # the extra blocks report their own failure instead of taking the headline line with
    # them; only rank 0 prints them, so only rank 0 runs them
    extra = rank == 0
    tte = None if args.no_time_to_energy or not extra else _block(time_to_energy, lem, pair, stream, tuned)
    more = {}
    if extra and not args.no_extra:
        more["middlebury_450x375"] = _block(middlebury_timing, lem, stream, flush)
        more["proposer"] = _block(proposer_timing, lem, stream)
        more["le_bf"] = _block(bf_timing, lem, workload_pair("middlebury_450x375", args.seed), stream, seed=31,
                               flush=flush, fp32_peak=peaks["fp32_tflops"])
        more["v3"] = _block(v3_timing, lem, stream, seed=41, flush=flush, pair=pair)

    if rank != 0:
        return
    value = world * evals_total / t_max
    # the dominant kernel's roofline: the data term's algorithmic FP32 work on the
    # batched-visit levels, else the data-term work of the whole iteration over the
    # one-kernel expansion time
    fp32_peak = peaks["fp32_tflops"]
    dk = kinds[dom]
    flops_launch = sum(work[l]["flops"] for l in dk["levels"]) / (dk["launches"] / args.steps)
    launch_ms = dk["ms"] / dk["launches"]
    achieved = flops_launch / (launch_ms / 1e3) / 1e12
    roof.update({"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                 "frac": achieved / fp32_peak, "traffic": traffic_from_profile(dom),
                 "launch_avg_ms": launch_ms, "flops_per_launch": flops_launch, "levels": dk["levels"],
                 "peak_note": "of measured: FP32 FMA throughput from lem_measure_peaks on this GPU",
                 "work_note": "algorithmic FP32 operations of the data term (30 per raw cost over M, 44 per "
                              "regression window, 24 per output pixel, per candidate and region) of the levels "
                              "this kernel runs"})
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "height": H, "width": W, "disp_max": DISP_MAX, "cells": pinfo["cell"],
                   "window": 4 * pinfo["gf_radius"] + 1, "store": "fp16 images, fp32 costs",
                   "candidates_per_visit": 4,
                   "step": "one outer iteration (3 levels x 16 groups, one dataflow launch per level)",
                   "iterations_per_handle": ITERS_PER_HANDLE, "l2": "flushed between timed steps",
                   "graph": "outer iterations replayed as CUDA graphs", "launch_config": tuning,
                   "parallelism": f"replicas x{world}", "evals_per_step": evals_per_step},
        "e2e": {"value": e2e_v, "unit": METRIC, "h2d_bytes_per_step": 2 * H * W * 3, "d2h_bytes_per_step": H * W * 4,
                "step": f"one job: host images -> lem_create -> {ITERS_PER_HANDLE} iterations -> host disparity",
                "jobs": args.e2e_jobs, "ms_per_job": 1e3 * e2e_job},
        # every expansion launch of the timed steps (counted from the library's events) and
        # the iteration-index kernel of each graph replay
        "gpu_launches": launches + graph_steps,
        "roofline": roof,
        "clocks": clk.summary(),
        "energy": {"first_handle_initial": e_first, "last_handle_final": e_last},
        "peaks": peaks,
    }
    if tte is not None:
        out["time_to_energy"] = tte
        if isinstance(tte, dict) and tte.get("learned_ms"):
            out["time_to_energy_ms"] = tte["learned_ms"]
            out["plain_ms"] = tte["plain_ms"]
            out["speedup"] = tte["speedup"]
    out.update(more)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = _block(cpu_oracle_baseline, pair, seed=1)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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


def _render(args):
    from synth import workload_pair
    seed, name = args
    p = workload_pair(name, seed)
    return {"left": p["left"], "right": p["right"]}


def run_cnn_gain_mode(args):
    """--mode cnn_gain: the learned proposer on held-out 1500 x 1000 scenes (seeds 100 ..
    100 + n - 1 of the headline workload; the network was trained on 384 x 288 scenes only).
    Per seed: E_plain after the plain method's 10 iterations (sequential proposals, FP32
    images); then, both with 4-candidate visits and FP16 images at one launch configuration,
    batched visits without and with learned proposals (k_cnn = 1 at the finest level) for up
    to 10 iterations each: time to E <= 1.001 E_plain, energy at equal wall-clock (the energy
    the run without the network has when the run with it reaches the target) and the share
    of switched pixels and of map candidates' moves that came from the network.  One JSON
    line with the per-seed records and their medians."""
    import multiprocessing as mp

    import numpy as np
    import torch

    import __graft_entry__
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    seeds = [100 + k for k in range(args.seeds)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        pairs = pool.map(_render, [(s, WORKLOAD) for s in seeds], chunksize=1)
    __graft_entry__.build()
    from paper_1603_08328_gb300 import lem, proposer
    stream = torch.cuda.current_stream()
    net = proposer.load()
    # one launch configuration for every run: tuned once on the first scene
    t = lem.Stereo(pairs[0]["left"], pairs[0]["right"], stream=stream, seed=5, **headline_params(lem))
    t.iterate(1, stats=False)
    tu = t.autotune(repeats=1)
    t.close()
    tuned = dict(level_threads=list(tu.threads), level_gr_interval=list(tu.gr_interval),
                 level_strip_rows=list(tu.strip_rows))

    def run(g, use_net, n):
        curve, t_ms, acc_map, acc_all = [], 0.0, 0, 0
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if use_net:
                g.cnn_propose(net)
            g.check(lem.lem_expand_iteration(g.h, 1, None))
            b.record(stream)
            b.synchronize()
            t_ms += a.elapsed_time(b)
            st = g.iterate(0)
            acc_all += st.accepted
            acc_map += st.accepted_by_kind[2]
            curve.append((st.energy, t_ms))
        return curve, acc_map, acc_all

    recs = []
    for s, pr in zip(seeds, pairs):
        g = lem.Stereo(pr["left"], pr["right"], stream=stream, seed=s, disp_max=DISP_MAX)
        g.iterate(1, stats=False)
        g.iterate(ITERS_PER_HANDLE - 1, stats=False)
        e_plain = g.energy()[0]
        g.close()
        target = 1.001 * e_plain
        fast = dict(headline_params(lem), seed=s, **tuned)
        g = lem.Stereo(pr["left"], pr["right"], stream=stream, **fast)
        base, _, acc_b = run(g, False, ITERS_PER_HANDLE)
        g.close()
        g = lem.Stereo(pr["left"], pr["right"], stream=stream, k_cnn=(1, 0, 0), **fast)
        cnn, acc_map, acc_c = run(g, True, ITERS_PER_HANDLE)
        g.close()

        def first(curve):
            for k, (e, tt) in enumerate(curve):
                if e <= target:
                    return k + 1, tt
            return None, None

        bi, bt = first(base)
        ci, ct = first(cnn)
        # energy at equal wall-clock: the run without the network at the time the run with
        # it reached the target (its last iteration finished by then)
        e_base_at = None
        if ct is not None:
            done = [e for e, tt in base if tt <= ct]
            e_base_at = done[-1] if done else None
        recs.append({"seed": s, "e_plain": e_plain, "batched_ms": bt, "batched_iters": bi, "cnn_ms": ct,
                     "cnn_iters": ci, "speedup": (bt / ct) if (bt and ct) else None,
                     "e_cnn_at_target": cnn[ci - 1][0] if ci else None, "e_batched_at_same_time": e_base_at,
                     "cnn_share_of_switches": acc_map / max(1, acc_c),
                     "e_after_2": {"batched": base[1][0], "cnn": cnn[1][0]}})
    net.close()
    sp = [r["speedup"] for r in recs if r["speedup"]]
    gain2 = [r["e_after_2"]["batched"] - r["e_after_2"]["cnn"] for r in recs]
    out = {"mode": "cnn_gain", "workload": WORKLOAD, "seeds": seeds,
           "config": {"plain": "sequential proposals, FP32 images, 10 iterations -> E_plain",
                      "batched": "4-candidate visits, FP16 images", "learned": "batched + k_cnn = (1, 0, 0)",
                      "launch_config": tuned},
           "median_speedup": float(np.median(sp)) if sp else None,
           "seeds_reaching_target": {"batched": sum(1 for r in recs if r["batched_ms"]),
                                     "cnn": sum(1 for r in recs if r["cnn_ms"])},
           "median_energy_gain_after_2_iterations": float(np.median(gain2)),
           "median_cnn_share_of_switches": float(np.median([r["cnn_share_of_switches"] for r in recs])),
           "per_seed": recs}
    print(json.dumps(out), flush=True)


def run_block_mode(args):
    """--mode v3 / lebf: one of the extra blocks of the default run on its own."""
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
    else:
        out = bf_timing(lem, workload_pair("middlebury_450x375", args.seed), stream, seed=31, flush=flush)
    print(json.dumps({"mode": args.mode, **out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode in ("v3", "lebf"):
        run_block_mode(args)
    elif args.mode == "proposer":
        run_proposer_mode(args)
    elif args.mode == "batch8":
        run_batch8_mode(args)
    elif args.mode == "cnn_gain":
        run_cnn_gain_mode(args)
    else:
        run_lem(args)


if __name__ == "__main__":
    main()
