"""The shell's per-ray merge on the GPU (ocr_fold_segments, the device
function the shell render runs per ray) against the oracle's compositing
rule, on lists with real overlaps (Sec. 2.5: where segments overlap, the ray
is cut at every segment end, each covering segment cut to the piece with Eq.
2.20, the covering pieces averaged with Eq. 2.21, the pieces combined with
Eq. 2.14).  In a valid forest only rounding slivers overlap, so the render
alone never exercises this branch with pieces large enough to matter.  The
expected values are built from the oracle's pinned cut, average and combine.
"""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


def _expected(vals, ivs):
    """The oracle's rule: elementary intervals between segment ends, near to
    far; the covering segments' pieces averaged, then combined nearest first."""
    pts = np.unique(ivs.reshape(-1))
    acc = np.array([1.0, 0.0, 0.0, 0.0])
    for lo, hi in zip(pts[:-1], pts[1:]):
        cov = [k for k in range(len(vals)) if ivs[k, 0] <= lo and ivs[k, 1] >= hi]
        if not cov:
            continue
        pieces = [O.cut(vals[k], (hi - lo) / (ivs[k, 1] - ivs[k, 0])) for k in cov]
        p = pieces[0]
        for q in pieces[1:]:  # at most two cover a piece in these lists
            p = O.average(p, q)
        acc = O.combine(acc, p)
    return acc


def _run(vals, ivs):
    from paper_1809_01334_gb300 import capi
    v = torch.from_numpy(vals.astype(np.float32)).cuda()
    iv = torch.from_numpy(ivs.astype(np.float32)).cuda()
    out = torch.zeros(4, device="cuda")
    capi.fold_segments(v, iv, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _values(rng, n):
    return np.column_stack([rng.uniform(0.3, 0.95, n), rng.uniform(0.0, 0.5, (n, 3))])


@pytest.mark.parametrize("n", [1, 5, 40, 100])
def test_disjoint_segments_fold_in_order(n):
    rng = np.random.default_rng(n)
    vals = _values(rng, n)
    ends = np.cumsum(rng.uniform(0.5, 2.0, 2 * n)) + 1.0
    ivs = ends.reshape(n, 2)
    got, ref = _run(vals, ivs), _expected(vals, ivs)
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-6)


@pytest.mark.parametrize("kind", ["partial", "contained", "equal", "mixed"])
def test_overlapping_pairs_are_cut_and_averaged(kind):
    """Isolated pairs of overlapping segments (each overlap between two
    segments, the next segment starting after the pair ends), between
    disjoint ones: the device's pairwise resolution is the oracle's rule."""
    rng = np.random.default_rng({"partial": 1, "contained": 2, "equal": 3, "mixed": 4}[kind])
    vals, ivs, x = [], [], 1.0
    for k in range(24):
        kk = kind if kind != "mixed" else ["partial", "contained", "equal", "none"][k % 4]
        a0 = x
        a1 = a0 + rng.uniform(1.0, 2.0)
        if kk == "partial":
            b0 = a0 + rng.uniform(0.2, 0.8) * (a1 - a0)
            pair = [(a0, a1), (b0, a1 + rng.uniform(0.3, 1.5))]
        elif kk == "contained":
            b0 = a0 + rng.uniform(0.1, 0.4) * (a1 - a0)
            pair = [(a0, a1), (b0, b0 + rng.uniform(0.1, 0.5) * (a1 - b0))]
        elif kk == "equal":
            pair = [(a0, a1), (a0 + 1e-3 * (a1 - a0), a1)]
        else:
            pair = [(a0, a1)]
        for p in pair:
            ivs.append(p)
        vals.append(_values(rng, len(pair)))
        x = max(p[1] for p in pair) + rng.uniform(0.0, 0.5)
    vals = np.vstack(vals)
    ivs = np.array(ivs)
    got, ref = _run(vals, ivs), _expected(vals, ivs)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-6)
    # the overlaps matter: folding the same list as if disjoint is far off
    plain = np.array([1.0, 0.0, 0.0, 0.0])
    for v in vals:
        plain = O.combine(plain, v)
    assert np.abs(plain - ref).max() > 1e-3


def test_bad_arguments_are_rejected():
    from paper_1809_01334_gb300 import capi
    v = torch.zeros((0, 4), device="cuda")
    iv = torch.zeros((0, 2), device="cuda")
    out = torch.zeros(4, device="cuda")
    with pytest.raises(capi.OcrError):
        capi.fold_segments(v, iv, out)
