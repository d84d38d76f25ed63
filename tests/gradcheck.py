"""Per-coordinate comparison of a GPU gradient with the FP64 oracle gradient.

The strict test on every coordinate is
    |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|).
A few coordinates can miss it without a fault:
  * cancellation: a coordinate is a sum of many terms (one per field
    evaluation touching it); where they cancel to far below their own size,
    the sum carries the FP32 rounding of the terms.  The oracle returns the
    sum of the terms' magnitudes (mag); for fixed-step integrators every
    coordinate outside the strict test must lie within 1e-4 mag of the
    oracle (about a thousand FP32 roundings of that scale).
  * adaptive step trees (DOPRI5 inside Algorithm 1): a split test near its
    threshold can go either way in FP32 and FP64, and the two sides then
    differentiate two different, equally valid discretisations; the oracle's
    own gradient moves as much on those coordinates when its tolerance is
    lowered a hundredfold.
At most max_frac of the coordinates (at least one) may miss the strict test,
and each of them by no more than abs_frac of the largest gradient entry.
"""
import numpy as np


def check(g, g_ref, what, mag=None, max_frac=1e-4, abs_frac=1e-4):
    g = np.asarray(g, np.float64).reshape(-1)
    r = np.asarray(g_ref, np.float64).reshape(-1)
    gmax = np.abs(r).max()
    scale = np.maximum(np.abs(r), 1e-3 * gmax)
    err = np.abs(g - r)
    miss = err > 1e-3 * scale
    n = int(miss.sum())
    worst = float((err[miss] / gmax).max()) if n else 0.0
    assert n <= max(1, max_frac * g.size), (
        f"{what}: {n} of {g.size} coordinates miss the strict test (worst {worst:.2e} max|g|)")
    assert worst <= abs_frac, (
        f"{what}: {n} coordinates miss the strict test, the worst by {worst:.2e} max|g|")
    if mag is not None:
        m = np.asarray(mag, np.float64).reshape(-1)
        unexplained = miss & (err > 1e-3 * scale + 1e-4 * m)
        assert not unexplained.any(), (
            f"{what}: {int(unexplained.sum())} coordinates beyond the rounding of their sums")
    return n
