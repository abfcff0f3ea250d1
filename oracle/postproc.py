"""Reference of the right-view estimate and the post-processing (test infrastructure only).

Right view.  The data term of the right image swaps the two images and adds the
disparity in the warp (Sec. 3.2, after Eq. photofunc).  Mirroring both images
horizontally turns that problem into the left-view one: the mirrored right image
becomes the reference and the mirrored left image the matched one, and a right
pixel u maps to u' = W - 1 - u.  A plane (a', b', c') found there is, in right-image
coordinates, a = -a', b = b', c = c' + a' (W - 1).

Post-processing (Sec. 3.4, end; the paper follows Bleyer et al. 2011 and is silent on
the details, so these are the readings):
  1. left-right consistency: a left pixel p with disparity d_L(p) is consistent when
     the right pixel q = (round(u - d_L(p)), v) lies in the image and
     |d_L(p) - d_R(q)| <= 1;
  2. filling: an inconsistent pixel takes, of the nearest consistent pixels to its
     left and right on the same row, the plane that gives the lower disparity at the
     pixel (occlusions are filled from the background); with one side only, that one;
  3. weighted median: every inconsistent pixel's disparity becomes the weighted median
     of the filled disparities in the (2 r + 1)^2 window around it (clipped to the
     image), weights exp(-|I_p - I_q|_1 / gamma) on the 0..255 left colours, r = 20
     (a 41 x 41 window) and gamma = 10; the weighted median is the smallest window
     value whose cumulative weight, in ascending order, reaches half the total.
Disparities are evaluated in FP32 as (a u + b v) + c, each operation rounded once,
so the consistency decisions are the same as in any FP32 evaluation in that order.
"""
from __future__ import annotations

import numpy as np


def mirror_planes_to_right(abc_m):
    """Planes found on the mirrored pair (H, W, 3) -> right-image planes (H, W, 3), in
    right-image pixel order."""
    abc_m = np.asarray(abc_m, np.float64)
    W = abc_m.shape[1]
    a, b, c = abc_m[..., 0], abc_m[..., 1], abc_m[..., 2]
    out = np.stack([-a, b, c + a * (W - 1)], axis=-1)
    return out[:, ::-1]


def disparity_f32(abc):
    """(a u + b v) + c in FP32, one rounding per operation."""
    abc = np.asarray(abc, np.float32)
    H, W = abc.shape[:2]
    v, u = np.mgrid[0:H, 0:W].astype(np.float32)
    return (abc[..., 0] * u + abc[..., 1] * v) + abc[..., 2]


def disparity_mirror_f32(abc_m):
    """Right-view disparity at right pixel u from the mirrored labels: the mirrored
    label at u' = W - 1 - u evaluated at u', in FP32."""
    d = disparity_f32(abc_m)
    return d[:, ::-1]


def lr_check(dL, dR, thr=1.0):
    """Consistency mask of the left view (rule 1)."""
    dL = np.asarray(dL, np.float32)
    dR = np.asarray(dR, np.float32)
    H, W = dL.shape
    u = np.arange(W, dtype=np.float32)[None, :]
    q = np.rint(u - dL)  # numpy rounds half to even, as rintf
    inside = (q >= 0) & (q <= W - 1)
    qi = np.clip(q, 0, W - 1).astype(np.int64)
    dq = np.take_along_axis(dR, qi, axis=1)
    return inside & (np.abs(dL - dq) <= np.float32(thr))


def fill_invalid(abcL, valid):
    """Rule 2: disparities (FP32) of the filled map."""
    abcL = np.asarray(abcL, np.float32)
    H, W = valid.shape
    d = disparity_f32(abcL)
    out = d.copy()
    for y in range(H):
        vrow = valid[y]
        for x in range(W):
            if vrow[x]:
                continue
            cands = []
            for step in (-1, 1):
                k = x + step
                while 0 <= k < W and not vrow[k]:
                    k += step
                if 0 <= k < W:
                    a, b, c = abcL[y, k]
                    cands.append((np.float32(a) * np.float32(x) + np.float32(b) * np.float32(y)) + np.float32(c))
            if cands:
                out[y, x] = min(cands)
    return out


def weighted_median(disp, valid, left, radius=20, gamma=10.0):
    """Rule 3 on the filled disparities; returns the final map (FP64 weights)."""
    disp = np.asarray(disp, np.float64)
    left = np.asarray(left, np.float64)
    H, W = disp.shape
    out = disp.copy()
    ys, xs = np.nonzero(~valid)
    for y, x in zip(ys, xs):
        y0, y1 = max(0, y - radius), min(H, y + radius + 1)
        x0, x1 = max(0, x - radius), min(W, x + radius + 1)
        vals = disp[y0:y1, x0:x1].ravel()
        wts = np.exp(-np.abs(left[y0:y1, x0:x1] - left[y, x]).sum(-1).ravel() / gamma)
        order = np.argsort(vals, kind="stable")
        cw = np.cumsum(wts[order])
        k = int(np.searchsorted(cw, 0.5 * cw[-1]))
        out[y, x] = vals[order[min(k, len(vals) - 1)]]
    return out


def is_weighted_median(value, vals, wts, rel=1e-5):
    """Whether `value` is a weighted median of (vals, wts) up to a relative weight
    tolerance: value is one of vals, the weight strictly below it is at most half the
    total and the weight up to and including it is at least half (both within rel)."""
    vals = np.asarray(vals, np.float64)
    wts = np.asarray(wts, np.float64)
    tot = wts.sum()
    if not np.any(vals == value):
        return False
    below = wts[vals < value].sum()
    upto = wts[vals <= value].sum()
    return below <= 0.5 * tot * (1 + rel) and upto >= 0.5 * tot * (1 - rel)
