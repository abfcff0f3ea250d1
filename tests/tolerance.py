"""Parity bar of the data term phi_p(f) against the FP64 oracle.

The bar is relative: |gpu - oracle| <= tol * |oracle|, tol = 1e-4 with FP32 image
storage and 2e-3 with FP16 / BF16 storage.

Below PHI_FLOOR = 0.1 the denominator is the floor, so there the bar is the absolute
tol * 0.1.  Why a floor: phi is a guided-filter mean of raw costs rho in [0, 2.8]
(Eq. photofunc) whose weights sum to one but may be negative (Eq. gf), so a small
phi can be the difference of terms near the top of that range, and the FP32 rounding
of those terms (a few 1e-7 of 2.8) is absolute, not relative to phi.  0.1 is the raw
cost of one gray level of colour mismatch between matched pixels (0.1 min(|dI|_1,
10)): costs below it are well inside the noise (sigma = 2 gray levels) of the inputs,
where a relative bar would measure the rounding of a cancellation rather than the
computation.
"""
import numpy as np

PHI_FLOOR = 0.1
PHI_TOL = 1e-4       # FP32 image storage
PHI_TOL_16 = 2e-3    # FP16 / BF16 image storage


def rel_err(gpu, ref):
    """|gpu - ref| / max(|ref|, PHI_FLOOR), elementwise, in FP64."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), PHI_FLOOR)


def report(label, gpu_list, ref_list):
    """Prints max and p99 of the relative error over all the results, the largest
    absolute error and how many oracle values lie below the floor; returns the max."""
    g = np.concatenate([np.asarray(x, np.float64).ravel() for x in gpu_list])
    r = np.concatenate([np.asarray(x, np.float64).ravel() for x in ref_list])
    e = rel_err(g, r)
    print(f"{label}: rel err max {e.max():.3e}, p99 {np.quantile(e, 0.99):.3e}, abs err max "
          f"{np.abs(g - r).max():.3e}, {int((np.abs(r) < PHI_FLOOR).sum())} of {r.size} below the floor")
    return float(e.max())
