"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test compares the oracle with something other than itself: a closed form,
a library routine, an invariant, or a brute-force evaluation of the defining
integral.  They are chosen so that a plausible slip anywhere in the oracle (a
dropped term, a wrong sign or index, a swapped operand, a mistyped tableau
entry) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1809_01334_gb300 import inputs as I
from tests import bruteforce as BF

RNG = np.random.default_rng(20180904)


def rand_seg(rng=RNG):
    return np.concatenate([[rng.uniform(0.05, 1.0)], rng.uniform(-1.0, 2.0, 3)])


# ---------------------------------------------------------------- Sec. 2.4 --
def test_combine_matches_sequential_application():
    """Eq. 2.14 with 2 = nearer: applying the far segment first and then the
    near one to an intensity (Eq. 2.11) equals applying their combination."""
    for _ in range(50):
        n, f = rand_seg(), rand_seg()
        Ib = RNG.uniform(-1, 1, 3)
        seq = n[0] * (f[0] * Ib + f[1:]) + n[1:]
        c = O.combine(n, f)
        np.testing.assert_allclose(c[0] * Ib + c[1:], seq, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(c[0], n[0] * f[0], rtol=1e-15)


def _all_bracketings(segs):
    if len(segs) == 1:
        yield segs[0]
        return
    for k in range(1, len(segs)):
        for left in _all_bracketings(segs[:k]):
            for right in _all_bracketings(segs[k:]):
                yield O.combine(left, right)


def test_combine_associative_under_every_bracketing():
    """Theorem of Sec. 2.4: the action is associative (all 42 bracketings of 6)."""
    segs = [rand_seg() for _ in range(6)]
    vals = np.array(list(_all_bracketings(segs)))
    assert vals.shape[0] == 42
    np.testing.assert_allclose(vals, np.broadcast_to(vals[0], vals.shape), rtol=1e-13, atol=1e-13)


def test_identity_inverse_and_non_commutativity():
    """Eq. 2.15: identity (1, 0), inverse (1/A, -B/A); the group is non-abelian."""
    e = np.array([1.0, 0, 0, 0])
    for _ in range(20):
        s = rand_seg()
        np.testing.assert_allclose(O.combine(e, s), s, rtol=1e-15)
        np.testing.assert_allclose(O.combine(s, e), s, rtol=1e-15)
        np.testing.assert_allclose(O.combine(s, O.inverse(s)), e, atol=1e-14)
        np.testing.assert_allclose(O.combine(O.inverse(s), s), e, atol=1e-14)
    a, b = np.array([0.5, 1.0, 0, 0]), np.array([0.25, 2.0, 0, 0])
    assert not np.allclose(O.combine(a, b), O.combine(b, a))


# ---------------------------------------------------------------- Sec. 2.5 --
def const_seg(beta, gamma, dx):
    """Eq. 2.13 (constant medium) with its beta -> 0 limit."""
    A = math.exp(-beta * dx)
    B = gamma * dx if beta == 0.0 else gamma / beta * -math.expm1(-beta * dx)
    return np.array([A, B, B * 0.5, B * 2.0])


@pytest.mark.parametrize("beta", [0.0, 1e-9, 0.3, 2.0, 15.0])
def test_cut_matches_constant_medium_and_recombines(beta):
    """Eq. 2.20: a cut piece equals the closed form on the shorter length, and
    near piece (+) far piece gives the whole segment back."""
    dx, gamma = 0.7, 1.3
    s = const_seg(beta, gamma, dx)
    for f in [0.0, 0.1, 0.5, 0.93, 1.0]:
        piece = O.cut(s, f)
        np.testing.assert_allclose(piece, const_seg(beta, gamma, f * dx), rtol=1e-12, atol=1e-15)
        rest = O.cut(s, 1.0 - f)
        np.testing.assert_allclose(O.combine(piece, rest), s, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(O.combine(rest, piece), s, rtol=1e-12, atol=1e-15)


def test_cut_transparent_special_case():
    """Eq. 2.20, A = 1: B_i = B dx_i / dx."""
    s = np.array([1.0, 0.8, 0.2, 0.4])
    np.testing.assert_allclose(O.cut(s, 0.25), [1.0, 0.2, 0.05, 0.1], rtol=1e-15)


def test_average_properties():
    """Eq. 2.21: idempotent, symmetric, geometric mean of A, arithmetic mean of B;
    for equal absorption it is the limit of finer and finer alternation of the
    two media (the construction in the proof of Sec. 2.5)."""
    for _ in range(10):
        s1, s2 = rand_seg(), rand_seg()
        np.testing.assert_allclose(O.average(s1, s1), s1, rtol=1e-15)
        np.testing.assert_allclose(O.average(s1, s2), O.average(s2, s1), rtol=1e-15)
    beta, dx = 1.7, 0.5
    s1, s2 = const_seg(beta, 0.4, dx), const_seg(beta, 2.2, dx)
    errs = []
    for N in (64, 256, 1024):
        p1, p2 = O.cut(s1, 0.5 / N), O.cut(s2, 0.5 / N)
        pair = O.combine(p2, p1)
        acc = np.array([1.0, 0, 0, 0])
        for _ in range(N):
            acc = O.combine(acc, pair)
        errs.append(np.abs(acc - O.average(s1, s2)).max())
    assert errs[2] < 5e-4 and errs[1] / errs[2] > 3.5  # first-order convergence
    # for unequal absorption the transmission of the alternation is exactly
    # the geometric mean at every N
    s1, s2 = const_seg(0.4, 0.4, dx), const_seg(6.0, 2.2, dx)
    for N in (1, 7, 64):
        pair = O.combine(O.cut(s2, 0.5 / N), O.cut(s1, 0.5 / N))
        acc = np.array([1.0, 0, 0, 0])
        for _ in range(N):
            acc = O.combine(acc, pair)
        assert abs(acc[0] - O.average(s1, s2)[0]) < 1e-14


# ------------------------------------------------------- field and TF --------
def test_tf_against_numpy_interp():
    f, tf, _, _ = I.preset_c1()
    of = O.OracleForest(f, tf)
    ss = np.concatenate([np.linspace(tf.s_min - 1, tf.s_max + 1, 101),
                         tf.s_min + np.arange(8) * (tf.s_max - tf.s_min) / 7])
    got = np.array([O.tf_eval(of, s) for s in ss])
    np.testing.assert_allclose(got, BF.tf_numpy(tf, ss), rtol=1e-13, atol=1e-13)


def test_trilinear_against_scipy_and_affine_exactness():
    from scipy.interpolate import RegularGridInterpolator
    vals = RNG.uniform(-2, 2, 8).astype(np.float32)
    rgi = RegularGridInterpolator(([0, 1], [0, 1], [0, 1]),
                                  vals.astype(np.float64).reshape(2, 2, 2).transpose(2, 1, 0))
    for _ in range(50):
        u = RNG.uniform(0, 1, 3)
        assert abs(O.trilinear(vals, *u) - rgi(u)[0]) < 1e-13
    # an affine function is reproduced exactly at any point
    a, b = 0.25, np.array([1.5, -2.0, 0.75])  # corner values exact in float32
    corners = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], float)
    nod = (a + corners @ b).astype(np.float32)
    for _ in range(20):
        u = RNG.uniform(-0.2, 1.2, 3)
        assert abs(O.trilinear(nod, *u) - (a + u @ b)) < 1e-12


# ------------------------------------------------------------- Sec. 2.2 -----
def test_ortho_rays_and_c1_rectangles():
    """C1 camera: ray (i, j) starts at ((i+1/2)/64, (j+1/2)/64, 3) and points
    down -z; leaf (a, b, c) of the level-3 grid covers pixels [8a, 8a+7] x
    [8b, 8b+7]."""
    f, tf, cam, _ = I.preset_c1()
    for i, j in [(0, 0), (5, 60), (63, 63)]:
        org, d, amin, amax = O.pixel_ray(cam, i, j)
        np.testing.assert_allclose(org, [(i + 0.5) / 64, (j + 0.5) / 64, 3.0], atol=1e-15)
        np.testing.assert_allclose(d, [0, 0, -1], atol=0)
    c = O.cull(f, tf, cam)
    assert c["visible"].all() and not c["uncertain"].any()
    a = f.anchor >> (f.max_level - 3)
    np.testing.assert_array_equal(c["rect"][:, 0], 8 * a[:, 0])
    np.testing.assert_array_equal(c["rect"][:, 1], 8 * a[:, 0] + 7)
    np.testing.assert_array_equal(c["rect"][:, 2], 8 * a[:, 1])
    np.testing.assert_array_equal(c["rect"][:, 3], 8 * a[:, 1] + 7)


def test_perspective_ray_reprojects_to_its_pixel():
    """Eq. 2.5 and Eq. 2.6 agree: the point o + r of pixel (i, j) lies on the
    projection plane (depth n) at pixel coordinates (i, j)."""
    cam = I.perspective_camera(7, 96, 54)
    t, u, v = (np.array(x) for x in (cam.t, cam.u, cam.v))
    for i, j in [(0, 0), (95, 53), (40, 17)]:
        org, d, amin, amax = O.pixel_ray(cam, i, j)
        assert amin == 1.0 and abs(amax - cam.far / cam.near) < 1e-9
        X = np.array([t @ d, u @ d, v @ d / cam.near])
        # t, u, v/n are orthonormal up to float32 rounding of the camera
        assert abs(X[2] - cam.near) < 1e-8
        pi = X[0] * cam.near / X[2] / cam.ell + (cam.w - 1) / 2
        pj = X[1] * cam.near / X[2] / cam.ell + (cam.h - 1) / 2
        assert abs(pi - i) < 1e-4 and abs(pj - j) < 1e-4


def test_rectangles_are_conservative_and_visibility_is_consistent():
    """Every ray that hits a leaf (brute-force pass over all pairs) lies in the
    leaf's pixel rectangle; a leaf hit by any ray is visible; invisible leaves
    are hit by no ray; a camera looking away sees nothing."""
    f, tf, cam = I.preset_small(w=40, h=30)
    of = O.OracleForest(f, tf)
    c = O.cull(f, tf, cam)
    hit_any = np.zeros(f.nleaves, bool)
    for j in range(cam.h):
        for i in range(cam.w):
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            for l in BF.leaves_along_ray(f, org, d, amin, amax):
                hit_any[l] = True
                r = c["rect"][l]
                assert r[0] <= i <= r[1] and r[2] <= j <= r[3]
    assert (c["visible"] | ~hit_any).all()
    assert c["visible"].sum() >= hit_any.sum()
    away = I.Camera(o=(0.5, 0.5, 3.0), v=(0.0, 0.0, 0.1), t=(1.0, 0, 0), u=(0, 1.0, 0),
                    ell=0.001, near=0.1, far=100.0, w=32, h=32)
    assert not O.cull(f, tf, away)["visible"].any()
    del of


def test_slab_chords_closed_form():
    """Chord lengths through the unit cube: 1 along an axis, sqrt(2) along a
    face diagonal, sqrt(3) along the body diagonal (one-leaf forest)."""
    fld = I.gaussian_field(4, 1809)
    f = I.uniform_cube_forest(0, fld)
    tf = I.transfer_function(f.nodal)
    of = O.OracleForest(f, tf)
    c = np.array([0.5, 0.5, 0.5])
    for d, L in [((0, 0, 1), 1.0), ((1, 1, 0), math.sqrt(2)), ((1, 1, 1), math.sqrt(3)),
                 ((-1, 1, -1), math.sqrt(3))]:
        d = np.array(d, float) * 0.37
        org = c - 5.0 * d
        hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0.0, 1e9)
        assert hit and abs((a1 - a0) * np.linalg.norm(d) - L) < 1e-14
    hit, _, _ = O.ray_leaf(of, 0, np.array([2.0, 0.5, 0.5]), np.array([0.0, 0.0, 1.0]), 0, 1e9)
    assert not hit


# ------------------------------------------------------------- Sec. 2.3/2.7 --
def _one_leaf(values, knots):
    fld = I.gaussian_field(4, 1809)
    f = I.uniform_cube_forest(0, fld)
    f.nodal = np.asarray(values, np.float32).reshape(1, 8)
    tf = I.TransferFunction(np.asarray(knots, np.float32), 0.0, 7.0)
    return f, tf


def _taylor4(z):
    return 1 - z + z * z / 2 - z ** 3 / 6 + z ** 4 / 24


@pytest.mark.parametrize("kappa", [0.5, 7.0, 19.0])
def test_rk4_constant_medium_is_taylor4(kappa):
    """Classical RK4 on A' = -k A, B' = q - k B from (1, 0) gives, per step,
    A = T4(k h) (degree-4 Taylor polynomial of exp(-k h)) and B = q/k (1 - A);
    four steps compose to A = T4^4, B = q/k (1 - T4^4)."""
    q = np.array([0.25, 0.5, 0.75])  # exact in float32
    knots = np.tile(np.concatenate([[kappa], q]), (8, 1))
    f, tf = _one_leaf(np.full(8, 3.0), knots)
    of = O.OracleForest(f, tf)
    d = np.array([0.3, -0.2, 1.0])
    org = np.array([0.5, 0.5, 0.5]) - 3.0 * d
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
    L = (a1 - a0) * np.linalg.norm(d)
    seg, steps = O.segment_ab(of, {"method": "rk4", "nsteps": 4}, 0, org, d, a0, a1)
    A = _taylor4(kappa * L / 4) ** 4
    np.testing.assert_allclose(seg[0], A, rtol=1e-13)
    np.testing.assert_allclose(seg[1:], q / kappa * (1 - A), rtol=1e-12)
    assert steps == 4


def test_transparent_medium_integrates_cubic_emission_exactly():
    """kappa = 0 and q linear in s: B = int q(s(x)) dx along the chord, with s
    trilinear (a cubic in x).  RK4 (Simpson weights) and DOPRI5 (order 5) both
    integrate it exactly; the reference is Gauss-Legendre quadrature."""
    vals = RNG.uniform(0.5, 6.5, 8)
    knots = np.zeros((8, 4))
    knots[:, 1] = np.arange(8) / 8.0      # q linear in s over [0, 7], knots exact in float32
    knots[:, 2] = 0.5
    knots[:, 3] = 0.75 - np.arange(8) / 16.0
    f, tf = _one_leaf(vals, knots)
    of = O.OracleForest(f, tf)
    d = np.array([0.4, 0.25, -0.9])
    org = np.array([0.45, 0.55, 0.5]) - 2.0 * d
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
    rl = np.linalg.norm(d)
    xg, wg = np.polynomial.legendre.leggauss(8)
    al = 0.5 * (a0 + a1) + 0.5 * (a1 - a0) * xg
    pts = org[None, :] + al[:, None] * d[None, :]
    s, _ = BF.field_at(f, pts)
    qv = BF.tf_numpy(tf, s)[:, 1:]
    ref = (wg[:, None] * qv).sum(0) * 0.5 * (a1 - a0) * rl
    for integ in ({"method": "rk4", "nsteps": 4},
                  {"method": "dopri5", "tol": 1.0, "c_rk": 1e9, "max_depth": 0}):
        seg, _ = O.segment_ab(of, integ, 0, org, d, a0, a1)
        assert seg[0] == 1.0
        np.testing.assert_allclose(seg[1:], ref, rtol=1e-13, atol=1e-14)
    # the embedded fourth-order solution (weights b*, seventh node c = 1) is
    # exact for a cubic integrand too, so the error estimate vanishes and a
    # tight tolerance causes no split
    seg, steps = O.segment_ab(of, {"method": "dopri5", "tol": 1e-13, "c_rk": 1e9,
                                   "max_depth": 8}, 0, org, d, a0, a1)
    assert steps == 1


def test_dopri5_single_step_is_fifth_order():
    """One DOPRI5 step on a constant medium (kappa dx = z) returns the method's
    stability polynomial R(-z) = sum_{k<=5} (-z)^k/k! + z^6/600, so
    R - exp(-z) = z^6 (1/600 - 1/720) + O(z^7) = z^6/3600 + O(z^7).  The z^6
    coefficient involves every entry of the tableau."""
    errs = []
    zs = (0.125, 0.0625, 0.03125)
    for z in zs:
        knots = np.tile([z, 0.0, 0.0, 0.0], (8, 1))
        f, tf = _one_leaf(np.full(8, 1.0), knots)
        of = O.OracleForest(f, tf)
        org, d = np.array([0.5, 0.5, -1.0]), np.array([0.0, 0.0, 1.0])
        seg, st = O.segment_ab(of, {"method": "dopri5", "tol": 1.0, "c_rk": 1e9, "max_depth": 0},
                               0, org, d, 1.0, 2.0)
        assert st == 1
        errs.append(seg[0] - math.exp(-z))
    assert 55 < errs[0] / errs[1] < 72 and 58 < errs[1] / errs[2] < 68
    assert abs(errs[2] / zs[2] ** 6 * 3600 - 1) < 0.04


def test_adaptive_bisection_tree_and_closed_form():
    """Algorithm 1 with the stability test only: a constant medium of optical
    depth k L splits uniformly to depth d = ceil(log2(k L / c_RK)), evaluating
    2^(d+1) - 1 steps; with a tight tolerance the result converges to the
    closed form exp(-k L), (q/k)(1 - exp(-k L))."""
    kappa, q = 12.0, np.array([0.25, 0.5, 0.875])  # exact in float32
    knots = np.tile(np.concatenate([[kappa], q]), (8, 1))
    f, tf = _one_leaf(np.full(8, 2.0), knots)
    of = O.OracleForest(f, tf)
    org, d = np.array([0.5, 0.5, -1.0]), np.array([0.0, 0.0, 1.0])
    c_rk = 0.5
    seg, steps = O.segment_ab(of, {"method": "dopri5", "tol": 1e9, "c_rk": c_rk, "max_depth": 30},
                              0, org, d, 1.0, 2.0)
    depth = math.ceil(math.log2(kappa * 1.0 / c_rk))
    assert steps == 2 ** (depth + 1) - 1
    seg, _ = O.segment_ab(of, {"method": "dopri5", "tol": 1e-13, "c_rk": 0.5, "max_depth": 30},
                          0, org, d, 1.0, 2.0)
    A = math.exp(-kappa)
    np.testing.assert_allclose(seg, np.concatenate([[A], q / kappa * (1 - A)]), rtol=1e-10)


def test_reversal_gives_the_inverse():
    """Sec. 2.6: running a segment backwards with negated coefficients gives
    the inverse, so the two combine to the identity (DOPRI5, tight tol)."""
    vals = RNG.uniform(0.5, 6.5, 8)
    knots = np.column_stack([RNG.uniform(0, 8, 8), RNG.uniform(0, 1, (8, 3))])
    f, tf = _one_leaf(vals, knots)
    fn, tfn = _one_leaf(vals, -knots)
    of, ofn = O.OracleForest(f, tf), O.OracleForest(fn, tfn)
    d = np.array([0.3, 0.5, -0.8])
    org = np.array([0.5, 0.45, 0.55]) - 2.0 * d
    integ = {"method": "dopri5", "tol": 1e-12, "c_rk": 0.5, "max_depth": 30}
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
    fwd, _ = O.segment_ab(of, integ, 0, org, d, a0, a1)
    org_r = org + (a0 + a1) * d  # same chord, opposite direction
    hit, b0, b1 = O.ray_leaf(ofn, 0, org_r, -d, 0, 1e9)
    assert abs((b1 - b0) - (a1 - a0)) < 1e-12
    back, _ = O.segment_ab(ofn, integ, 0, org_r, -d, b0, b1)
    np.testing.assert_allclose(O.combine(back, fwd), [1, 0, 0, 0], atol=1e-9)
    np.testing.assert_allclose(O.combine(fwd, back), [1, 0, 0, 0], atol=1e-9)


# ------------------------------------------------------------ brute force ----
def _tiny(level, seed=1809):
    fld = I.gaussian_field(4, seed)
    f = I.uniform_cube_forest(level, fld)
    tf = I.transfer_function(f.nodal, 1334, kappa_max=8.0)
    return f, tf


@pytest.mark.parametrize("level", [0, 1, 2])
def test_render_matches_quadrature_of_the_closed_form(level):
    """Whole-image brute force on 1, 8 and 64 leaves: per ray, the closed-form
    solution (Eq. 2.12) by trapezoid quadrature on 2e5 points with point
    location -- no segments, no sorting, no group action -- against the oracle
    with a fine discretisation; the configured RK4 x 4 stays within its
    truncation error.  Includes a non-zero background."""
    f, tf = _tiny(level)
    cam = I.perspective_camera(11 + level, 8, 6, dist=(1.8, 2.2))
    bg = (0.2, 0.1, 0.05)
    # the FP64 definition (decide32=False): rays and intervals in FP64, as the
    # quadrature below takes them
    fine = O.render(f, tf, cam, {"method": "dopri5", "tol": 1e-12, "c_rk": 0.1, "max_depth": 30},
                    bg=bg, decide32=False)
    coarse = [O.render(f, tf, cam, {"method": "rk4", "nsteps": n}, bg=bg, decide32=False)["rgba"]
              for n in (4, 8)]
    ref = np.zeros((cam.h, cam.w, 4))
    for j in range(cam.h):
        for i in range(cam.w):
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            ref[j, i] = BF.ray_integral(f, tf, org, d, amin, amax, bg=bg)
    assert (fine["counts"] > 0).sum() > 10
    np.testing.assert_allclose(fine["rgba"], ref, atol=2e-8)
    # the configured RK4 differs from the exact solution by its truncation
    # error; the transfer function's kinks limit RK4 to second order locally,
    # with a constant that depends on where a kink falls in a step, so only a
    # bound and a decrease with more steps are asserted (the one-leaf chord
    # has k h up to 2.6 per step at 4 steps)
    e4, e8 = (np.abs(c - ref).max() for c in coarse)
    assert e4 < (0.05 if level == 0 else 2e-3) and e8 < e4


@pytest.mark.parametrize("kind", ["uniform2", "adaptive"])
def test_segment_counts_match_point_location(kind):
    """Per-ray segment counts equal the number of leaves a ray passes, found
    by point location between finest-level plane crossings."""
    f, tf, cam = I.preset_small(kind=kind, w=24, h=20)
    r = O.render(f, tf, cam, {"method": "rk4", "nsteps": 1})
    for j in range(cam.h):
        for i in range(cam.w):
            if r["uncertain"][j, i]:
                continue
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            assert r["counts"][j, i] == len(BF.leaves_along_ray(f, org, d, amin, amax))


def test_c1_counts_and_alpha():
    """C1: every ray of the orthographic 64x64 image crosses the 8 leaves of
    its column; the image is opaque-ish but not fully (alpha < 1)."""
    f, tf, cam, integ = I.preset_c1()
    r = O.render(f, tf, cam, integ)
    assert (r["counts"] == 8).all() and r["segments"] == 64 * 64 * 8
    assert (r["rgba"][..., 3] > 0).all() and (r["rgba"][..., 3] < 1).all()


def test_overlapping_segments_are_cut_and_averaged():
    """Sec. 2.5: where segments overlap, the ray is cut at their ends and the
    overlapping pieces are averaged.  (1) Two leaves on the same box with
    different data: the pixel is the average of the two single-leaf pixels.
    (2) A leaf covering the near half of another: the pixel is the far half of
    the big leaf (+) ... built from the separately pinned cut/average/combine."""
    fld = I.gaussian_field(4, 1809)
    base = I.uniform_cube_forest(0, fld, max_level=1)
    v1 = RNG.uniform(0.0, 1.0, 8).astype(np.float32)
    v2 = RNG.uniform(0.0, 1.0, 8).astype(np.float32)
    tf = I.TransferFunction(np.column_stack([np.linspace(0.5, 6, 8), RNG.uniform(0, 1, (8, 3))])
                            .astype(np.float32), 0.0, 1.0)
    cam = I.Camera(o=(0.5, 0.5, 3.0), v=(0.0, 0.0, -1.0), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                   ell=0.25, near=1.0, far=1e30, w=4, h=4, ortho=True)
    integ = {"method": "rk4", "nsteps": 16}

    def forest(levels, anchors, nodal):
        return I.Forest("cube", 1, np.array(levels, np.uint8), np.array(anchors, np.int32),
                        np.zeros(len(levels), np.int32), np.array(nodal, np.float32))

    one1 = O.render(forest([0], [[0, 0, 0]], [v1]), tf, cam, integ)["rgba"]
    one2 = O.render(forest([0], [[0, 0, 0]], [v2]), tf, cam, integ)["rgba"]
    both = O.render(forest([0, 0], [[0, 0, 0], [0, 0, 0]], [v1, v2]), tf, cam, integ)
    assert (both["counts"] == 2).all()
    exp_alpha = 1.0 - np.sqrt((1.0 - one1[..., 3]) * (1.0 - one2[..., 3]))
    np.testing.assert_allclose(both["rgba"][..., 3], exp_alpha, rtol=1e-13)
    np.testing.assert_allclose(both["rgba"][..., :3], 0.5 * (one1[..., :3] + one2[..., :3]),
                               rtol=1e-13)
    # partial overlap: big leaf [0,1]^3 and small leaf [0,1/2]^3 (the near half
    # of the big one along -z lies at z in [1/2, 1], so use anchor z = 1)
    f2 = forest([0, 1], [[0, 0, 0], [0, 0, 1]], [v1, v2])
    of2 = O.OracleForest(f2, tf)
    r = O.render(f2, tf, cam, integ)
    for i, j in [(0, 0), (1, 1), (1, 0)]:
        org, d, amin, amax = O.pixel_ray(cam, i, j)
        _, a0, a1 = O.ray_leaf(of2, 0, org, d, amin, amax)
        _, b0, b1 = O.ray_leaf(of2, 1, org, d, amin, amax)
        assert abs(a0 - b0) < 1e-15 and b1 < a1
        big, _ = O.segment_ab(of2, integ, 0, org, d, a0, a1)
        small, _ = O.segment_ab(of2, integ, 1, org, d, b0, b1)
        fr = (b1 - b0) / (a1 - a0)
        near = O.average(O.cut(big, fr), small)
        tot = O.combine(near, O.cut(big, 1.0 - fr))
        np.testing.assert_allclose(r["rgba"][j, i], np.concatenate([tot[1:], [1 - tot[0]]]),
                                   rtol=1e-12)


# ------------------------------------------------ Sec. 2.7: Gauss-2, Simpson --
@pytest.mark.parametrize("kappa", [0.5, 7.0, 19.0])
def test_gauss2_constant_medium_is_pade22(kappa):
    """Eqs. 2.32-2.33 on a constant medium: A is the (2,2) Pade approximant of
    exp(-z), z = k dx, and B = (q/k)(1 - A)."""
    q = np.array([0.25, 0.5, 0.75])
    f, tf = _one_leaf(np.full(8, 3.0), np.tile(np.concatenate([[kappa], q]), (8, 1)))
    of = O.OracleForest(f, tf)
    org, d = np.array([0.5, 0.5, -1.0]), np.array([0.0, 0.0, 1.0])
    seg, st = O.segment_ab(of, {"method": "gauss2", "c_rk": 1e9, "max_depth": 0}, 0, org, d,
                           1.0, 2.0)
    z = kappa
    A = (1 - z / 2 + z * z / 12) / (1 + z / 2 + z * z / 12)
    assert st == 1
    np.testing.assert_allclose(seg, np.concatenate([[A], q / kappa * (1 - A)]), rtol=1e-13)


def test_gauss2_equals_direct_gauss_legendre_solve():
    """On a varying medium one Gauss-2 step equals the two-stage Gauss-Legendre
    method (c = 1/2 -+ sqrt(3)/6 from the far end, A = [[1/4, 1/4 - sqrt(3)/6],
    [1/4 + sqrt(3)/6, 1/4]], b = (1/2, 1/2)) solved as a linear system."""
    vals = RNG.uniform(0.5, 6.5, 8)
    knots = np.column_stack([RNG.uniform(0, 8, 8), RNG.uniform(0, 1, (8, 3))])
    f, tf = _one_leaf(vals, knots)
    of = O.OracleForest(f, tf)
    d = np.array([0.3, -0.4, 0.85])
    org = np.array([0.5, 0.5, 0.5]) - 2.0 * d
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
    seg, _ = O.segment_ab(of, {"method": "gauss2", "c_rk": 1e9, "max_depth": 0}, 0, org, d, a0, a1)
    r3 = math.sqrt(3.0)
    c = np.array([0.5 - r3 / 6, 0.5 + r3 / 6])
    Ag = np.array([[0.25, 0.25 - r3 / 6], [0.25 + r3 / 6, 0.25]])
    rl = np.linalg.norm(d)
    H = (a1 - a0) * rl
    al = a1 - c * H / rl  # x = c H from the far end
    s, _ = BF.field_at(f, org[None, :] + al[:, None] * d[None, :])
    kq = BF.tf_numpy(tf, s)
    beta, gam = kq[:, 0], kq[:, 1:]
    # stages k_i = g_i - beta_i (y0 + H sum_j A_ij k_j): (I + H diag(beta) A) k = g - beta y0
    M = np.eye(2) + H * beta[:, None] * Ag
    kA = np.linalg.solve(M, -beta * 1.0)
    ref = [1.0 + H * kA.sum() / 2]
    for ch in range(3):
        kB = np.linalg.solve(M, gam[:, ch])
        ref.append(H * kB.sum() / 2)
    np.testing.assert_allclose(seg, ref, rtol=1e-12, atol=1e-14)


def test_simpson_exact_for_cubic_media():
    """Eq. 2.34: Simpson's rule integrates cubics exactly, so with kappa and q
    linear in the trilinear field (cubic along the ray) A = exp(-int kappa)
    exactly, and with kappa = 0, B = int q exactly (Gauss-Legendre reference)."""
    vals = RNG.uniform(0.5, 6.5, 8)
    xg, wg = np.polynomial.legendre.leggauss(8)
    d = np.array([0.35, 0.2, -0.9])
    org = np.array([0.5, 0.45, 0.5]) - 2.0 * d
    for kap_knots, q_r in [(np.arange(8) / 4.0, np.full(8, 0.5)),
                           (np.zeros(8), np.arange(8) / 8.0)]:
        knots = np.column_stack([kap_knots, q_r, np.full(8, 0.25), np.full(8, 0.125)])
        f, tf = _one_leaf(vals, knots)
        of = O.OracleForest(f, tf)
        hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
        seg, _ = O.segment_ab(of, {"method": "simpson", "c_rk": 1e9, "max_depth": 0}, 0, org, d,
                              a0, a1)
        al = 0.5 * (a0 + a1) + 0.5 * (a1 - a0) * xg
        s, _ = BF.field_at(f, org[None, :] + al[:, None] * d[None, :])
        kq = BF.tf_numpy(tf, s)
        L = (a1 - a0) * np.linalg.norm(d)
        tau = (wg * kq[:, 0]).sum() * 0.5 * L
        np.testing.assert_allclose(seg[0], math.exp(-tau), rtol=1e-13)
        if not kap_knots.any():
            np.testing.assert_allclose(seg[1], (wg * kq[:, 1]).sum() * 0.5 * L, rtol=1e-13)


@pytest.mark.parametrize("method", ["gauss2", "simpson"])
def test_gauss2_simpson_converge_inside_algorithm1(method):
    """Inside Algorithm 1 both converge to the closed form of a constant medium
    as c_RK shrinks (Gauss at rate c_RK^4, Simpson's B at c_RK^2 or better),
    and split uniformly into 2^(d+1) - 1 evaluated steps."""
    kappa, q = 12.0, np.array([0.25, 0.5, 0.875])
    f, tf = _one_leaf(np.full(8, 2.0), np.tile(np.concatenate([[kappa], q]), (8, 1)))
    of = O.OracleForest(f, tf)
    org, d = np.array([0.5, 0.5, -1.0]), np.array([0.0, 0.0, 1.0])
    exact = np.concatenate([[math.exp(-kappa)], q / kappa * -math.expm1(-kappa)])
    errs = []
    for c_rk in (0.5, 0.25, 0.125):
        seg, st = O.segment_ab(of, {"method": method, "c_rk": c_rk, "max_depth": 30}, 0, org, d,
                               1.0, 2.0)
        depth = math.ceil(math.log2(kappa / c_rk))
        assert st == 2 ** (depth + 1) - 1
        errs.append(np.abs(seg - exact).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[1] / errs[2] > (12 if method == "gauss2" else 3.5)


# ------------------------------------------------- Eq. 2.18 as an interface --
def test_equilibrium_interface_constant_medium_is_exact():
    """Eq. 2.18: with constant kappa and intensity I the step is exactly the
    equilibrium solution, A = exp(-kappa L), B = I (1 - A), whatever the
    splitting (Eq. 2.13 with q = kappa I); every split gives the same value."""
    kappa, inten = 7.0, np.array([0.25, 0.5, 0.875])
    f, tf = _one_leaf(np.full(8, 2.0), np.tile(np.concatenate([[kappa], inten]), (8, 1)))
    of = O.OracleForest(f, tf)
    org, d = np.array([0.5, 0.5, -1.0]), np.array([0.0, 0.0, 1.0])
    L = 1.0
    exact = np.concatenate([[math.exp(-kappa * L)], inten * -math.expm1(-kappa * L)])
    for c_rk, depth in [(1e9, 0), (0.5, 30), (0.01, 30)]:
        seg, st = O.segment_ab(of, {"method": "equilibrium", "c_rk": c_rk, "max_depth": depth},
                               0, org, d, 1.0, 2.0)
        np.testing.assert_allclose(seg, exact, rtol=1e-12, atol=1e-15)
    # the same as the ODE of Eq. 2.29 with emission q = kappa I (fine DOPRI5)
    f2, tf2 = _one_leaf(np.full(8, 2.0), np.tile(np.concatenate([[kappa], kappa * inten]), (8, 1)))
    ode, _ = O.segment_ab(O.OracleForest(f2, tf2), {"method": "dopri5", "tol": 1e-12, "c_rk": 0.05,
                                                     "max_depth": 30}, 0, org, d, 1.0, 2.0)
    np.testing.assert_allclose(ode, exact, rtol=1e-10, atol=1e-12)


def test_equilibrium_interface_converges_to_the_ode_with_emission_kappa_times_intensity():
    """With varying data, Algorithm 1 with the Eq. 2.18 step converges, as
    c_RK shrinks, to Eq. 2.12 with q(x) = kappa(x) I(x): trapezoid quadrature
    of the closed form with point location (no segments) along the ray."""
    vals = RNG.uniform(0.5, 6.5, 8)
    knots = np.column_stack([1.0 + np.arange(8), 0.1 + 0.1 * np.arange(8),
                             0.9 - 0.1 * np.arange(8), np.full(8, 0.4)])
    f, tf = _one_leaf(vals, knots)
    of = O.OracleForest(f, tf)
    d = np.array([0.35, 0.2, -0.9])
    org = np.array([0.5, 0.45, 0.5]) - 2.0 * d
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0, 1e9)
    rl = np.linalg.norm(d)
    xs = np.linspace(0.0, (a1 - a0) * rl, 400001)
    pts = org[None, :] + (a1 - xs / rl)[:, None] * d[None, :]
    s, _ = BF.field_at(f, pts)
    kq = BF.tf_numpy(tf, s)
    kap, q = kq[:, 0], kq[:, :1] * kq[:, 1:]
    dx = xs[1] - xs[0]
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * dx)])
    fB = q * np.exp(-(tau[-1] - tau))[:, None]
    ref = np.concatenate([[math.exp(-tau[-1])], (0.5 * (fB[1:] + fB[:-1]) * dx).sum(axis=0)])
    errs = []
    for c_rk in (0.2, 0.05, 0.0125):
        seg, _ = O.segment_ab(of, {"method": "equilibrium", "c_rk": c_rk, "max_depth": 30}, 0,
                              org, d, a0, a1)
        errs.append(np.abs(seg - ref).max())
    # second order (I at the step midpoint): each 4x finer c_RK divides the error by ~16
    assert errs[2] < errs[1] < errs[0] and errs[2] < 2e-7 and errs[1] / errs[2] > 10, errs


# ------------------------------------------------------- Sec. 2.8 surfaces --
def _surface_case(a_s, nodal, kappa=3.0, inten=(0.2, 0.5, 0.9), c=(1, 2, 0.5), s_iso=0.5):
    f, tf = _one_leaf(nodal, np.tile(np.concatenate([[kappa], inten]), (8, 1)))
    of = O.OracleForest(f, tf)
    d = np.array(c, float)
    d /= np.linalg.norm(d) * 2.0
    org = np.array([0.43, 0.52, 0.55]) - 4.0 * d  # off the leaf's centre: no sample on the plane
    hit, a0, a1 = O.ray_leaf(of, 0, org, d, 0.0, 1e9)
    assert hit
    integ = {"method": "equilibrium", "c_rk": 1e9, "max_depth": 0,
             "surface": {"s_iso": s_iso, "a_s": a_s, "i_s": (0.7, 0.1, 0.3)}}
    seg, _ = O.segment_ab(of, integ, 0, org, d, a0, a1)
    return seg, org, d, a0, a1, kappa, np.asarray(inten, np.float32).astype(np.float64)


def _const_piece(kappa, inten, L):
    A = math.exp(-kappa * L)
    return np.concatenate([[A], inten * (1.0 - A)])


@pytest.mark.parametrize("plane", ["x", "y+2z"])
def test_planar_isosurface_closed_form(plane):
    """Eq. 2.35 on a plane (the isosurface 1/2 of the field s = x, or of
    s = (y + 2z)/4 at 3/8, whose normal is (0, 1, 2)/sqrt 5) inside a constant medium:
    the segment is near piece (+) surface (+) far piece, the surface with
    A = a_s^(1/cos phi), phi between the ray and the normal, and B = I_s (1 - A)
    (Eq. 2.18)."""
    if plane == "x":
        nodal = [float(c & 1) for c in range(8)]  # s = u_x
        nrm, iso = np.array([1.0, 0.0, 0.0]), 0.5
    else:
        nodal = [(((c >> 1) & 1) + 2.0 * ((c >> 2) & 1)) / 4.0 for c in range(8)]  # exact in float32
        nrm, iso = np.array([0.0, 1.0, 2.0]) / math.sqrt(5.0), 0.375
    for a_s in (0.0, 0.35, 0.9):
        seg, org, d, a0, a1, kappa, inten = _surface_case(a_s, nodal, s_iso=iso)
        rl = np.linalg.norm(d)
        # crossing of the plane n . x = n . (1/2, 1/2, 1/2)
        ac = (nrm @ np.full(3, 0.5) - nrm @ org) / (nrm @ d)
        assert a0 < ac < a1
        near = _const_piece(kappa, inten, (ac - a0) * rl)
        far = _const_piece(kappa, inten, (a1 - ac) * rl)
        cphi = abs(nrm @ d) / rl
        A = a_s ** (1.0 / cphi)
        surf = np.concatenate([[A], np.array([0.7, 0.1, 0.3]) * (1.0 - A)])
        exp = O.combine(near, O.combine(surf, far))
        np.testing.assert_allclose(seg, exp, rtol=1e-10, atol=1e-12)


def test_transparent_surface_is_invisible_and_opaque_surface_hides_the_rest():
    """a_s = 1 leaves the segment unchanged (B_s = I_s (1 - 1) = 0); a_s = 0
    makes everything behind the surface invisible."""
    nodal = [float(c & 1) for c in range(8)]
    seg1, org, d, a0, a1, kappa, inten = _surface_case(1.0, nodal)
    rl = np.linalg.norm(d)
    np.testing.assert_allclose(seg1, _const_piece(kappa, inten, (a1 - a0) * rl), rtol=1e-12)
    seg0, *_ = _surface_case(0.0, nodal)
    ac = (0.5 - org[0]) / d[0]
    near = _const_piece(kappa, inten, (ac - a0) * rl)
    assert seg0[0] == 0.0
    np.testing.assert_allclose(seg0[1:], near[1:] + near[0] * np.array([0.7, 0.1, 0.3]),
                               rtol=1e-12)


def test_two_crossings_and_none():
    """s = (2x - 1)(2y - 1) vanishes on the planes x = 1/2 and y = 1/2: a ray
    crossing both inside the leaf meets the isosurface s = 0 twice, in order;
    a ray through a region where s keeps its sign meets it never."""
    nodal = [(2 * (c & 1) - 1) * (2 * ((c >> 1) & 1) - 1) * 1.0 for c in range(8)]
    f, tf = _one_leaf(nodal, np.tile([2.0, 0.2, 0.5, 0.9], (8, 1)))
    tf.s_min, tf.s_max = -1.0, 1.0
    cam = I.Camera(o=(0.37, 0.61, 3.0), v=(0.0, 0.0, -1.0), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                   ell=0.125, near=1.0, far=1e30, w=4, h=4, ortho=True)
    surf = {"method": "equilibrium", "c_rk": 1e9, "max_depth": 0,
            "surface": {"s_iso": 0.0, "a_s": 0.5, "i_s": (1.0, 1.0, 1.0)}}
    r = O.render(f, tf, cam, surf)
    # orthographic rays along -z never cross the planes x = 1/2, y = 1/2
    assert (r["crossings"] == 0).all()
    of = O.OracleForest(f, tf)
    d = np.array([0.8, 0.9, 0.1])
    org = np.array([0.05, 0.1, 0.45])
    hit, a0, a1 = O.ray_leaf(of, 0, org - d, d, 0.0, 1e9)
    seg, _ = O.segment_ab(of, dict(surf, surface=dict(surf["surface"], a_s=0.0)), 0, org - d, d,
                          a0, a1)
    # an opaque surface: only the volume before the first crossing (x = 1/2 at
    # alpha 1 + 0.45/0.8, y = 1/2 at 1 + 0.4/0.9) and the surface's intensity
    first = 1.0 + min(0.45 / 0.8, 0.4 / 0.9)
    near = _const_piece(2.0, np.array([0.2, 0.5, 0.9], np.float32).astype(float),
                        (first - a0) * np.linalg.norm(d))
    np.testing.assert_allclose(seg, [0.0, *(near[1:] + near[0])], rtol=1e-10)


# ------------------------------------------------------- gradient (reverse) --
def _loss(forest, tf, cam, integ, W, bg):
    r = O.render(forest, tf, cam, integ, bg=bg)
    return float((r["rgba"] * W).sum()), r["steps"]


@pytest.mark.parametrize("integ", [{"method": "rk4", "nsteps": 4},
                                   {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16},
                                   {"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
                                   {"method": "simpson", "c_rk": 0.2, "max_depth": 16},
                                   {"method": "equilibrium", "c_rk": 0.2, "max_depth": 16}])
@pytest.mark.parametrize("part", ["knots", "nodal"])
def test_oracle_gradient_matches_central_differences(integ, part):
    """The FP64 reverse-mode gradient of L = sum(W * rgba) equals central
    differences of the (pinned) forward oracle.  Knots: all 32 knot values with
    the seeded transfer function (L is smooth in them).  Nodal values: with a
    transfer function linear in s (a piecewise-linear one makes L only
    piecewise smooth in s, which central differences cannot resolve).
    Perturbations are applied to the float32 inputs, the step is the exactly
    representable difference, and a coordinate whose perturbation changes the
    adaptive step tree is skipped (the gradient is that of the fixed tree)."""
    fld = I.gaussian_field(4, 7)
    f = I.uniform_cube_forest(1, fld)
    tf = I.transfer_function(f.nodal, 3, kappa_max=8.0)
    if part == "nodal":
        k = np.arange(8)
        tf.knots[:] = np.column_stack([0.5 + k, 0.1 + 0.1 * k, 0.8 - 0.1 * k, 0.3 + 0.05 * k])
        span = float(f.nodal.max() - f.nodal.min())  # keep every s inside the knot range
        tf.s_min, tf.s_max = float(f.nodal.min()) - 0.5 * span, float(f.nodal.max()) + 0.5 * span
    cam = I.perspective_camera(5, 8, 6, dist=(1.8, 2.2))
    bg = (0.2, 0.1, 0.05)
    rng = np.random.default_rng(11)
    W = rng.uniform(-1, 1, (cam.h, cam.w, 4))
    gn, gt = O.render_grad(f, tf, cam, integ, W, bg=bg)
    assert np.abs(gn).max() > 0 and np.abs(gt).max() > 0
    if part == "knots":
        coords, arr, g = range(32), tf.knots.reshape(-1), gt.reshape(-1)
    else:
        coords, arr, g = rng.choice(f.nodal.size, 24, replace=False), f.nodal.reshape(-1), gn.reshape(-1)
    scale = np.abs(g).max()
    checked = 0
    for k in coords:
        v = float(arr[k])
        h = 1e-3 * max(1.0, abs(v))
        vp, vm = np.float32(v + h), np.float32(v - h)
        arr[k] = vp
        lp, sp = _loss(f, tf, cam, integ, W, bg)
        arr[k] = vm
        lm, sm = _loss(f, tf, cam, integ, W, bg)
        arr[k] = np.float32(v)
        if sp != sm:
            continue
        fd = (lp - lm) / (float(vp) - float(vm))
        assert abs(g[k] - fd) <= 2e-5 * abs(fd) + 1e-6 * scale, (part, k, g[k], fd)
        checked += 1
    assert checked >= (28 if part == "knots" else 20)


def test_gradient_term_magnitudes():
    """The oracle's per-coordinate sum of term magnitudes (the scale of a
    gradient sum's rounding): never below the sum's own magnitude, unchanged
    when dL/d(rgba) changes sign (the gradient flips), linear in its scale,
    and equal to |g| where every term has one sign (dL/d alpha only, with a
    transfer function rising in kappa and constant in q: all terms of
    dL/d(nodal) then share the sign of the slope)."""
    f = I.uniform_cube_forest(1, I.gaussian_field(4, 7))
    tf = I.transfer_function(f.nodal, 3, kappa_max=8.0)
    cam = I.perspective_camera(5, 8, 6, dist=(1.8, 2.2))
    integ = {"method": "rk4", "nsteps": 4}
    W = np.random.default_rng(2).uniform(-1, 1, (cam.h, cam.w, 4))
    gn, gt, an, at = O.render_grad(f, tf, cam, integ, W, magnitudes=True)
    assert (an >= np.abs(gn) * (1 - 1e-12)).all() and (at >= np.abs(gt) * (1 - 1e-12)).all()
    assert an.max() > np.abs(gn).max()  # some terms cancel
    gn2, gt2, an2, at2 = O.render_grad(f, tf, cam, integ, -2.0 * W, magnitudes=True)
    np.testing.assert_allclose(gn2, -2.0 * gn, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(an2, 2.0 * an, rtol=1e-12, atol=1e-15)
    k = np.arange(8)
    tf.knots[:] = np.column_stack([0.5 + k, np.full(8, 0.3), np.full(8, 0.2), np.full(8, 0.1)])
    span = float(f.nodal.max() - f.nodal.min())
    tf.s_min, tf.s_max = float(f.nodal.min()) - span, float(f.nodal.max()) + span
    Wa = np.zeros((cam.h, cam.w, 4))
    Wa[..., 3] = 1.0
    gn, gt, an, at = O.render_grad(f, tf, cam, integ, Wa, magnitudes=True)
    assert np.abs(gn).max() > 0
    np.testing.assert_allclose(an, np.abs(gn), rtol=1e-6, atol=1e-15)
