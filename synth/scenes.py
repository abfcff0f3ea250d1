"""Seeded synthetic rectified stereo pairs.

This module is the one input generator that both the FP64 oracle and the CUDA
path consume.  It renders images only: it holds none of the stereo method's
arithmetic (no matching cost, filter, smoothness term or optimiser).

A scene lives in disparity space.  Every segment is a slanted plane
``d = a*u + b*v + c`` (optionally plus a quadric bump
``kappa*((u-u0)^2 + (v-v0)^2)``) with an elliptic support in left-view pixel
coordinates; one fronto-parallel background segment covers everything.  The
left view shows, at every pixel, the segment of largest disparity whose support
contains it (so occlusion boundaries are real).  Texture is multi-octave value
noise attached to each surface in left-view coordinates, so the right view is
an exact warp: right pixel (u_r, v) shows the surface point (u_l, v) with
``u_l - d(u_l, v) = u_r`` (closed form for planes, Newton for quadrics, keeping converged roots), again
taking the nearest (largest-disparity) surface.  Gaussian noise (sigma in gray
levels) is added independently to both views before rounding to uint8.

Disparity convention (left view): a left pixel u matches right pixel u - d.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Segment:
    a: float
    b: float
    c: float
    kappa: float          # quadric curvature (0 for a plane)
    u0: float             # bump / ellipse centre
    v0: float
    rx: float             # ellipse radii (inf for the background)
    ry: float
    theta: float          # ellipse orientation
    tex: "_ValueNoise"

    def disparity(self, u, v):
        d = self.a * u + self.b * v + self.c
        if self.kappa != 0.0:
            d = d + self.kappa * ((u - self.u0) ** 2 + (v - self.v0) ** 2)
        return d

    def ddu(self, u, v):
        g = np.full_like(u, self.a, dtype=np.float64)
        if self.kappa != 0.0:
            g = g + 2.0 * self.kappa * (u - self.u0)
        return g

    def inside(self, u, v):
        if not np.isfinite(self.rx):
            return np.ones(np.broadcast(u, v).shape, dtype=bool)
        ct, st = np.cos(self.theta), np.sin(self.theta)
        du, dv = u - self.u0, v - self.v0
        x = (ct * du + st * dv) / self.rx
        y = (-st * du + ct * dv) / self.ry
        return x * x + y * y <= 1.0


class _ValueNoise:
    """Colour value noise: lattice values blended with a smoothstep, summed over octaves."""

    def __init__(self, rng: np.random.Generator, umin, umax, vmin, vmax, base, contrast,
                 spacings=(24.0, 12.0, 6.0, 3.0)):
        self.octaves = []
        self.base = np.asarray(base, dtype=np.float64)
        amp = 1.0
        for sp in spacings:
            nu = int(np.ceil((umax - umin) / sp)) + 3
            nv = int(np.ceil((vmax - vmin) / sp)) + 3
            # partially correlated channels so the colour covariance is full rank
            common = rng.uniform(-1.0, 1.0, size=(nv, nu, 1))
            indep = rng.uniform(-1.0, 1.0, size=(nv, nu, 3))
            vals = 0.6 * common + 0.4 * indep
            self.octaves.append((sp, amp, vals, umin - sp, vmin - sp))
            amp *= 0.55
        self.contrast = contrast

    def __call__(self, u, v):
        out = np.zeros(np.broadcast(u, v).shape + (3,), dtype=np.float64)
        for sp, amp, vals, u_org, v_org in self.octaves:
            x = (u - u_org) / sp
            y = (v - v_org) / sp
            x = np.clip(x, 0.0, vals.shape[1] - 1.000001)
            y = np.clip(y, 0.0, vals.shape[0] - 1.000001)
            i = np.floor(x).astype(np.int64)
            j = np.floor(y).astype(np.int64)
            fx = x - i
            fy = y - j
            fx = fx * fx * (3.0 - 2.0 * fx)
            fy = fy * fy * (3.0 - 2.0 * fy)
            v00 = vals[j, i]
            v01 = vals[j, i + 1]
            v10 = vals[j + 1, i]
            v11 = vals[j + 1, i + 1]
            top = v00 + (v01 - v00) * fx[..., None]
            bot = v10 + (v11 - v10) * fx[..., None]
            out += amp * (top + (bot - top) * fy[..., None])
        return self.base + self.contrast * out


def _make_scene(rng: np.random.Generator, H: int, W: int, dmin: float, dmax: float,
                n_planes: int, n_quadrics: int):
    span = dmax - dmin
    umin, umax = -dmax - 8.0, W + dmax + 8.0
    segs = []

    def texture():
        base = rng.uniform(70.0, 185.0, size=3)
        contrast = rng.uniform(35.0, 60.0)
        return _ValueNoise(rng, umin, umax, -8.0, H + 8.0, base, contrast)

    # fronto-parallel background at the far end of the range
    c_bg = dmin + 0.12 * span
    segs.append(Segment(0.0, 0.0, c_bg, 0.0, W / 2, H / 2, np.inf, np.inf, 0.0, texture()))
    n_total = n_planes + n_quadrics
    for k in range(n_total):
        quad = k >= n_planes
        u0 = rng.uniform(0.1 * W, 0.9 * W)
        v0 = rng.uniform(0.1 * H, 0.9 * H)
        scale = min(W, H)
        rx = rng.uniform(0.12, 0.35) * scale
        ry = rng.uniform(0.12, 0.35) * scale
        theta = rng.uniform(0.0, np.pi)
        # centre disparity in the nearer part of the range, slopes bounded so the
        # disparity stays inside [dmin, dmax] over the ellipse's bounding box
        d0 = dmin + rng.uniform(0.3, 0.85) * span
        rmax = max(rx, ry)
        room = min(d0 - dmin, dmax - d0) * 0.7
        smax = min(0.35, room / max(rmax, 1.0))
        a = rng.uniform(-smax, smax)
        b = rng.uniform(-smax, smax)
        kappa = 0.0
        if quad:
            # a bump toward the camera: disparity decreases away from (u0, v0)
            kappa = -rng.uniform(0.2, 0.6) * room / max(rmax * rmax, 1.0)
        c = d0 - a * u0 - b * v0
        segs.append(Segment(a, b, c, kappa, u0, v0, rx, ry, theta, texture()))
    return segs


def _window(s, H, W, right):
    """Row and column slices that contain every pixel the segment can cover in the
    left view, or (right=True) in the right view (its support shifted by its
    disparity range over the support's bounding box)."""
    if not np.isfinite(s.rx):
        return slice(0, H), slice(0, W)
    R = max(s.rx, s.ry) + 1.0
    v0, v1 = int(np.floor(s.v0 - R)), int(np.ceil(s.v0 + R)) + 1
    u0, u1 = s.u0 - R, s.u0 + R
    if right:
        corners = [s.a * uu + s.b * vv + s.c for uu in (u0, u1) for vv in (s.v0 - R, s.v0 + R)]
        dhi = max(corners) + max(0.0, s.kappa) * 2.0 * R * R
        dlo = min(corners) + min(0.0, s.kappa) * 2.0 * R * R
        u0, u1 = u0 - dhi - 2.0, u1 - dlo + 2.0
    cu0, cu1 = int(np.floor(u0)), int(np.ceil(u1)) + 1
    return slice(max(0, v0), max(0, min(H, v1))), slice(max(0, cu0), max(0, min(W, cu1)))


def _render(segs, H, W):
    """Left view, right view (noise-free, float) and left ground-truth disparity.
    Each segment is evaluated only inside the window it can cover, and textures only
    at the pixels it wins."""
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    # left view: nearest segment containing the pixel
    best_d = np.full((H, W), -np.inf)
    best_s = np.zeros((H, W), dtype=np.int64)
    for k, s in enumerate(segs):
        ys, xs = _window(s, H, W, False)
        uu, vv = u[ys, xs], v[ys, xs]
        d = s.disparity(uu, vv)
        m = s.inside(uu, vv) & (d > best_d[ys, xs])
        best_d[ys, xs][m] = d[m]
        best_s[ys, xs][m] = k
    left = np.zeros((H, W, 3))
    for k, s in enumerate(segs):
        m = best_s == k
        if m.any():
            left[m] = s.tex(u[m], v[m])
    # right view: for each segment solve u_l - d(u_l, v) = u_r
    rbest = np.full((H, W), -np.inf)
    rseg = np.full((H, W), -1, dtype=np.int64)
    rul = np.zeros((H, W))
    for k, s in enumerate(segs):
        ys, xs = _window(s, H, W, True)
        uu, vv = u[ys, xs], v[ys, xs]
        ul = (uu + s.b * vv + s.c) / (1.0 - s.a)
        if s.kappa != 0.0:
            for _ in range(30):
                g = ul - s.disparity(ul, vv) - uu
                ul = ul - g / (1.0 - s.ddu(ul, vv))
        d = s.disparity(ul, vv)
        # a quadric's equation has a second root; Newton can also stall between
        # them: keep only solutions that satisfy the warp equation
        ok = np.abs(ul - d - uu) < 1e-6
        m = s.inside(ul, vv) & ok & (d > rbest[ys, xs])
        rbest[ys, xs][m] = d[m]
        rseg[ys, xs][m] = k
        rul[ys, xs][m] = ul[m]
    right = np.zeros((H, W, 3))
    for k, s in enumerate(segs):
        m = rseg == k
        if m.any():
            right[m] = s.tex(rul[m], v[m])
    return left, right, best_d


def make_pair(seed: int, height: int, width: int, disp_max: float, disp_min: float = 0.0,
              n_planes: int = 3, n_quadrics: int = 1, sigma: float = 2.0):
    """Render one seeded pair.

    Returns a dict with ``left`` and ``right`` (uint8, H x W x 3, RGB interleaved),
    ``disp`` (float64 left ground-truth disparity) and the scene parameters.
    """
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), height, width]))
    segs = _make_scene(rng, height, width, float(disp_min), float(disp_max), n_planes, n_quadrics)
    left, right, disp = _render(segs, height, width)
    noise_rng = np.random.default_rng(np.random.SeedSequence([int(seed), 7919]))
    if sigma > 0:
        left = left + noise_rng.normal(0.0, sigma, size=left.shape)
        right = right + noise_rng.normal(0.0, sigma, size=right.shape)
    left8 = np.clip(np.rint(left), 0, 255).astype(np.uint8)
    right8 = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return {"left": np.ascontiguousarray(left8), "right": np.ascontiguousarray(right8),
            "disp": disp, "segments": segs}


# Workload shapes (Middlebury-V2/V3-shaped synthetic stand-ins).
WORKLOADS = {
    # 96x72, disparities 0-15: 3 planes + 1 quadric bump over a fronto-parallel background
    "tiny_96x72": dict(height=72, width=96, disp_max=15.0, n_planes=3, n_quadrics=1),
    # 450x375, disparities 0-60, ~10 planar and quadric segments
    "middlebury_450x375": dict(height=375, width=450, disp_max=60.0, n_planes=7, n_quadrics=3),
    # 1500x1000, disparities 0-400, ~40 slanted and curved segments
    "large_1500x1000": dict(height=1000, width=1500, disp_max=400.0, n_planes=28, n_quadrics=12),
    # 384x288 training scenes for the proposal network
    "train_384x288": dict(height=288, width=384, disp_max=48.0, n_planes=7, n_quadrics=3),
}

# The uneven batch: 8 pairs from 640x480 to 2900x2000, disparity ranges 64-800 px.
BATCH8 = [
    dict(height=480, width=640, disp_max=64.0, n_planes=8, n_quadrics=3),
    dict(height=600, width=800, disp_max=96.0, n_planes=10, n_quadrics=4),
    dict(height=768, width=1024, disp_max=128.0, n_planes=14, n_quadrics=5),
    dict(height=960, width=1280, disp_max=192.0, n_planes=18, n_quadrics=6),
    dict(height=1000, width=1500, disp_max=256.0, n_planes=22, n_quadrics=8),
    dict(height=1080, width=1920, disp_max=400.0, n_planes=26, n_quadrics=10),
    dict(height=1600, width=2400, disp_max=600.0, n_planes=30, n_quadrics=12),
    dict(height=2000, width=2900, disp_max=800.0, n_planes=34, n_quadrics=14),
]


def workload_pair(name: str, seed: int = 0):
    return make_pair(seed, **WORKLOADS[name])


def batch8_pair(index: int, seed: int = 0):
    """Pair `index` (0..7) of the uneven batch."""
    return make_pair(seed * 8 + index, **BATCH8[index])


def _batch8_images(args):
    p = batch8_pair(*args)
    return {"left": p["left"], "right": p["right"], "disp": p["disp"]}


def render_batch8(seed: int = 0, processes: int = 8):
    """All 8 pairs of the uneven batch (left, right, disp), rendered in spawned
    worker processes (safe after CUDA has been initialised in the caller)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(processes) as pool:
        return pool.map(_batch8_images, [(i, seed) for i in range(len(BATCH8))], chunksize=1)


def random_labels(seed: int, n: int, height: int, width: int, disp_max: float,
                  slope: float = 0.5):
    """Random plane labels (a, b, c) as float32 rows, for parity tests of the cost path.

    Disparities at the image centre fall in [0, disp_max]; slopes in [-slope, slope].
    """
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 4242]))
    a = rng.uniform(-slope, slope, n)
    b = rng.uniform(-slope, slope, n)
    d = rng.uniform(0.0, disp_max, n)
    c = d - a * (width / 2.0) - b * (height / 2.0)
    return np.stack([a, b, c], axis=1).astype(np.float32)
