"""Per-coordinate comparison of a GPU gradient with the FP64 oracle gradient.

The strict test on every coordinate is
    |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|).
Two effects can make a coordinate miss it without a fault, and the allowance
for each is computed by the oracle, never taken from the GPU:
  * cancellation: a coordinate is a sum of many terms (one per field
    evaluation touching it); where they cancel to far below their own size,
    the sum carries the FP32 rounding of the terms.  The oracle returns the
    sum of the terms' magnitudes (mag); the allowance is 1e-4 mag, about a
    thousand FP32 roundings of that scale.
  * adaptive step trees (DOPRI5 inside Algorithm 1): a split test near its
    threshold can go either way in FP32 and FP64, and the two sides then
    differentiate two different (equally valid) discretisations.  The
    allowance is twice the oracle's own change of that coordinate when the
    tolerance is lowered a hundredfold (fine).
Every coordinate must pass the strict test or lie within the allowances, and
at most max_frac of them may need an allowance.
"""
import numpy as np


def check(g, g_ref, what, mag=None, fine=None, max_frac=1e-4):
    g = np.asarray(g, np.float64).reshape(-1)
    r = np.asarray(g_ref, np.float64).reshape(-1)
    scale = np.maximum(np.abs(r), 1e-3 * np.abs(r).max())
    err = np.abs(g - r)
    strict = err <= 1e-3 * scale
    allow = 1e-3 * scale
    if mag is not None:
        allow = allow + 1e-4 * np.asarray(mag, np.float64).reshape(-1)
    if fine is not None:
        allow = allow + 2.0 * np.abs(r - np.asarray(fine, np.float64).reshape(-1))
    ok = err <= allow
    n_allow = int((~strict).sum())
    assert ok.all(), (f"{what}: {int((~ok).sum())} of {g.size} coordinates outside the "
                      f"allowance, worst err/allowance {float((err / allow).max()):.3e}")
    assert n_allow <= max(1, max_frac * g.size), (
        f"{what}: {n_allow} of {g.size} coordinates need an allowance")
    return n_allow
