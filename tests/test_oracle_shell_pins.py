"""Pins of the FP64 oracle's cubed-sphere shell (six trees, the equiangular
map, degree-2 nodal data) to closed forms, invariants and brute force.

The brute-force side (tests/bruteforce.py) locates points by the face their
central projection lands on and inverts the map in NumPy; it never uses the
oracle's cone/sphere intersection, its culling bound, or its segments.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1809_01334_gb300 import inputs as I
from tests import bruteforce as BF

RNG = np.random.default_rng(1809_01334)


def _shell(level_min, level_max, theta=1e9, kappa_max=8.0):
    f = I.shell_forest(I.shell_noise(1809, 8), level_min, level_max, theta)
    tf = I.transfer_function(f.nodal, 1334, kappa_max=kappa_max)
    return f, tf


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------- the map --
def test_equiangular_map_closed_forms_and_inverse():
    """|x| = r(zeta); the tree centre maps to r n; tree corners map to the cube
    corners (n +- e1 +- e2)/sqrt(3); along eta = 1/2 the angle from n is
    pi/4 |2 xi - 1| (equal angles for equal steps); the inverse map undoes the
    map; the map agrees with the input generator's independent NumPy map."""
    f, tf = _shell(0, 0)
    of = O.OracleForest(f, tf)
    fr = np.asarray(f.meta["frames"])
    r0, r1 = f.meta["r0"], f.meta["r1"]
    for t in range(6):
        n, e1, e2 = fr[t]
        x = O.shell_map(of, t, [0.5, 0.5, 0.25])
        np.testing.assert_allclose(x, (r0 + 0.25 * (r1 - r0)) * n, atol=1e-15)
        for a, b in [(0, 0), (0, 1), (1, 0), (1, 1)]:
            x = O.shell_map(of, t, [a, b, 1.0])
            np.testing.assert_allclose(x, r1 * _unit(n + (2 * a - 1) * e1 + (2 * b - 1) * e2),
                                       atol=1e-15)
        for xi in np.linspace(0, 1, 9):
            x = O.shell_map(of, t, [xi, 0.5, 0.0])
            ang = math.acos(min(1.0, float(x @ n) / r0))
            assert abs(ang - math.pi / 4 * abs(2 * xi - 1)) < 1e-12
        for _ in range(20):
            ref = RNG.uniform(0, 1, 3)
            x = O.shell_map(of, t, ref)
            assert abs(np.linalg.norm(x) - (r0 + ref[2] * (r1 - r0))) < 1e-14
            np.testing.assert_allclose(O.shell_inverse(of, t, x), ref, atol=1e-13)
            np.testing.assert_allclose(x, I.shell_map(t, *ref), atol=1e-14)


def test_six_trees_tile_the_sphere():
    """Every direction belongs to exactly one tree: the inverse map of exactly
    one tree with x . n > 0 lands in [0, 1]^2 (away from tree boundaries)."""
    f, tf = _shell(0, 0)
    of = O.OracleForest(f, tf)
    fr = np.asarray(f.meta["frames"])
    for _ in range(300):
        x = _unit(RNG.normal(size=3)) * 0.8
        owners = []
        for t in range(6):
            if x @ fr[t, 0] <= 0:
                continue
            ref = O.shell_inverse(of, t, x)
            if np.all((ref[:2] >= 0) & (ref[:2] <= 1)):
                owners.append((t, ref))
        assert owners, x
        margins = [min(np.min(r[:2]), np.min(1 - r[:2])) for _, r in owners]
        assert len(owners) == 1 or min(margins) < 1e-9, [t for t, _ in owners]


def test_triquadratic_nodes_and_polynomial_exactness():
    """Lagrange property at the 27 nodes (index a + 3 b + 9 c at (a, b, c)/2),
    exact reproduction of any product of quadratics, partition of unity."""
    for c in range(27):
        e = np.zeros(27, np.float32)
        e[c] = 1.0
        for k in range(27):
            v = O.triquadratic(e, (k % 3) / 2, ((k // 3) % 3) / 2, (k // 9) / 2)
            assert v == (1.0 if k == c else 0.0)
    p = lambda u, v, w: (1 + u - 2 * v * v + u * v * w + 0.5 * u * u * v * v * w * w
                         - 0.25 * w * w * u)
    nod = np.array([p((k % 3) / 2, ((k // 3) % 3) / 2, (k // 9) / 2) for k in range(27)],
                   np.float32)
    for _ in range(50):
        u, v, w = RNG.uniform(-0.2, 1.2, 3)
        assert abs(O.triquadratic(nod, u, v, w) - p(u, v, w)) < 1e-5  # float32 nodal values
    ones = np.ones(27, np.float32)
    for _ in range(10):
        assert abs(O.triquadratic(ones, *RNG.uniform(0, 1, 3)) - 1.0) < 1e-14


# ----------------------------------------------------------- ray ∩ shell leaf --
def _all_intervals(of, f, org, d, amin=0.0, amax=1e9):
    out = []
    for l in range(f.nleaves):
        iv, _ = O.ray_leaf_intervals(of, l, org, d, amin, amax)
        out.extend((a, b, l) for a, b in iv)
    return sorted(out)


def test_radial_rays_closed_form():
    """A ray from 3u towards the centre meets the leaf around u on
    alpha in [3 - R_out, 3 - R_in] and the leaf around -u on
    [3 + R_in, 3 + R_out] (unit direction); all other leaves are missed."""
    f, tf = _shell(2, 2)
    of = O.OracleForest(f, tf)
    r0, r1 = f.meta["r0"], f.meta["r1"]
    for _ in range(10):
        u = _unit(RNG.normal(size=3))
        iv = _all_intervals(of, f, 3.0 * u, -u)
        # level 2: four radial layers on each side of the centre
        assert len(iv) == 8
        radii = r0 + (r1 - r0) * np.arange(5) / 4
        near = [3.0 - r for r in radii[::-1]]
        far = [3.0 + r for r in radii]
        exp = [(near[k], near[k + 1]) for k in range(4)] + [(far[k], far[k + 1]) for k in range(4)]
        for (a, b, _), (ea, eb) in zip(iv, exp):
            assert abs(a - ea) < 1e-12 and abs(b - eb) < 1e-12


def test_leaf_chords_tile_the_shell_chord():
    """For random lines, the leaves' intervals do not overlap and their total
    length is the chord of the annulus: 2 sqrt(r1^2 - p^2) - 2 sqrt(r0^2 - p^2)
    (second term only if p < r0), p the line's distance from the centre.
    Adaptive unbalanced forest, levels 1..3."""
    f, tf, _ = I.preset_shell_small()
    of = O.OracleForest(f, tf)
    r0, r1 = f.meta["r0"], f.meta["r1"]
    for k in range(12):
        d = _unit(RNG.normal(size=3)) * RNG.uniform(0.5, 2.0)
        p = RNG.uniform(-1, 1, 3) * (0.3 if k < 6 else 0.95)
        p -= (p @ d) / (d @ d) * d
        org = p - 4.0 * d
        iv = _all_intervals(of, f, org, d)
        pl = np.linalg.norm(p)
        if pl >= r1:
            assert not iv
            continue
        L = 2 * math.sqrt(r1 * r1 - pl * pl) - (2 * math.sqrt(r0 * r0 - pl * pl) if pl < r0 else 0)
        tot = sum((b - a) for a, b, _ in iv) * np.linalg.norm(d)
        assert abs(tot - L) < 1e-12
        for (a0, b0, _), (a1, b1, _) in zip(iv, iv[1:]):
            assert a1 >= b0 - 1e-12


def test_intervals_match_point_location():
    """Per-leaf intervals against membership by point location (the tree from
    the face of the central projection, the leaf from the inverse map) at
    dense samples along the ray; the ray through the hollow of a level-0 tree
    gets two intervals of the same leaf."""
    f, tf, _ = I.preset_shell_small()
    of = O.OracleForest(f, tf)
    for k in range(8):
        d = _unit(RNG.normal(size=3))
        p = RNG.uniform(-1, 1, 3) * 0.7
        p -= (p @ d) * d
        org = p - 3.0 * d
        iv = _all_intervals(of, f, org, d)
        al = np.linspace(1.0, 5.0, 40001)
        leaf, _ = BF.shell_locate(f, org[None, :] + al[:, None] * d[None, :])
        got = np.full(al.shape, -1)
        for a, b, l in iv:
            got[(al > a) & (al < b)] = l
        # samples within 1e-9 of an interval end may go either way
        ends = np.array([x for a, b, _ in iv for x in (a, b)] or [np.inf])
        far = np.min(np.abs(al[:, None] - ends[None, :]), axis=1) > 1e-9
        assert (got[far] == leaf[far]).all()
    f0, tf0 = _shell(0, 0)
    of0 = O.OracleForest(f0, tf0)
    # the line x = 0.5, z = 0 along y crosses tree +x, and the hollow for
    # |y| < sqrt(0.55^2 - 0.25)
    org, d = np.array([0.5, -2.0, 0.0]), np.array([0.0, 1.0, 0.0])
    t = int(np.argmax(np.asarray(f0.meta["frames"])[:, 0, 0]))
    iv, _ = O.ray_leaf_intervals(of0, t, org, d, 0.0, 10.0)
    y = math.sqrt(0.55 ** 2 - 0.25)
    exp = [(1.5, 2.0 - y), (2.0 + y, 2.5)]
    assert len(iv) == 2
    for (a, b), (ea, eb) in zip(iv, exp):
        assert abs(a - ea) < 1e-12 and abs(b - eb) < 1e-12


def test_segment_counts_match_boundary_crossings():
    """Per-ray segment counts of the oracle render equal the number of leaf
    visits found by point location between all crossings of the finest
    level's boundary planes and spheres (adaptive shell, perspective)."""
    f, tf, cam = I.preset_shell_small(w=20, h=16)
    r = O.render(f, tf, cam, {"method": "rk4", "nsteps": 1})
    checked = 0
    for j in range(cam.h):
        for i in range(cam.w):
            if r["uncertain"][j, i]:
                continue
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            assert r["counts"][j, i] == len(BF.shell_leaves_along_ray(f, org, d, amin, amax))
            checked += 1
    assert checked > 0.9 * cam.w * cam.h and r["counts"].max() >= 8


# ------------------------------------------------------------------ culling --
@pytest.mark.parametrize("case", ["adaptive", "level0"])
def test_shell_rectangles_contain_the_projected_leaf(case):
    """The culling bound (corner AABB widened by r_out (1 - cos phi)) holds
    the projection of every point of the leaf: dense samples of each leaf,
    mapped by the input generator's map, project inside the projected
    extents; and the bound is not loose by more than a small factor.  The
    six 90-degree leaves of a level-0 shell bulge far beyond their corners."""
    if case == "adaptive":
        f, tf, cam = I.preset_shell_small(w=40, h=32)
        leaves = RNG.choice(f.nleaves, 150, replace=False)
    else:
        f, tf = _shell(0, 0)
        cam = I.perspective_camera(21, 40, 32, dist=(3.0, 3.5), target=(0.0, 0.0, 0.0))
        leaves = range(6)
    of = O.OracleForest(f, tf)
    g = np.linspace(0, 1, 9)
    U = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    t_, u_, v_ = (np.asarray(a, float) for a in (cam.t, cam.u, cam.v))
    o = np.asarray(cam.o, float)
    worst = 0.0
    for l in leaves:
        vis, rect, pext, _ = O.leaf_rect(of, cam, l)
        h = 2.0 ** -int(f.level[l])
        ref = f.anchor[l] / float(1 << f.max_level) + U * h
        x = I.shell_map(np.full(len(U), f.tree[l]), ref[:, 0], ref[:, 1], ref[:, 2])
        X = np.stack([(x - o) @ t_, (x - o) @ u_, (x - o) @ v_ / cam.near], -1)
        assert (X[:, 2] > cam.near).all()  # the small preset sits in front of the camera
        pi = X[:, 0] * cam.near / X[:, 2] / cam.ell + (cam.w - 1) / 2
        pj = X[:, 1] * cam.near / X[:, 2] / cam.ell + (cam.h - 1) / 2
        assert (pi >= pext[0] - 1e-9).all() and (pi <= pext[1] + 1e-9).all()
        assert (pj >= pext[2] - 1e-9).all() and (pj <= pext[3] + 1e-9).all()
        span = max(pi.max() - pi.min(), pj.max() - pj.min())
        worst = max(worst, (pext[1] - pext[0]) / max(span, 1e-9))
        if vis:
            inside = ((pi >= -0.5) & (pi <= cam.w - 0.5) & (pj >= -0.5) & (pj <= cam.h - 0.5))
            assert inside.any() or rect[1] >= rect[0]
    assert worst < (2.0 if case == "adaptive" else 3.0)


def test_shell_rectangles_are_conservative_for_rays():
    """Every pixel whose ray meets a leaf (oracle intervals) lies in the
    leaf's rectangle, and the leaf is visible."""
    f, tf, cam = I.preset_shell_small(w=24, h=20)
    of = O.OracleForest(f, tf)
    c = O.cull(f, tf, cam)
    for j in range(0, cam.h, 3):
        for i in range(0, cam.w, 3):
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            for l in BF.shell_leaves_along_ray(f, org, d, amin, amax):
                r = c["rect"][l]
                assert c["visible"][l] and r[0] <= i <= r[1] and r[2] <= j <= r[3]


# ------------------------------------------------------------------- render --
def test_constant_field_closed_form():
    """Constant nodal values give constant kappa, q: every pixel is
    A = exp(-kappa L), B = q (1 - A) / kappa with L the ray's chord through
    the annulus, over a background."""
    f, tf, cam = I.preset_shell_small(w=16, h=12)
    f.nodal[:] = np.float32(0.3)
    tf.s_min, tf.s_max = -1.0, 1.0
    bg = (0.3, 0.2, 0.1)
    r = O.render(f, tf, cam, {"method": "dopri5", "tol": 1e-10, "c_rk": 0.2, "max_depth": 30},
                 bg=bg, decide32=False)  # the FP64 definition, as the closed form below
    kq = BF.tf_numpy(tf, np.array([0.3]))[0]
    for j in range(cam.h):
        for i in range(cam.w):
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            L = sum(b - a for a, b in BF.shell_pieces(f, org, d, amin, amax)) * np.linalg.norm(d)
            A = math.exp(-kq[0] * L)
            exp = [A * bg[c] + kq[1 + c] * (1 - A) / kq[0] for c in range(3)] + [1 - A]
            np.testing.assert_allclose(r["rgba"][j, i], exp, atol=1e-9)
    assert (r["rgba"][..., 3] > 0).sum() > 40


@pytest.mark.parametrize("level", [1, 2])
def test_shell_render_matches_quadrature_of_the_closed_form(level):
    """Uniform shells (48 and 384 leaves, the field continuous across leaf
    faces): per ray, the closed-form solution (Eq. 2.12) by trapezoid
    quadrature on each piece inside the shell, with point location and the
    degree-2 interpolation written in NumPy, against the oracle with a fine
    discretisation."""
    f, tf = _shell(level, level)
    cam = I.perspective_camera(3 + level, 8, 6, dist=(2.0, 2.4), target=(0.0, 0.0, 0.0))
    bg = (0.2, 0.1, 0.05)
    fine = O.render(f, tf, cam, {"method": "dopri5", "tol": 1e-12, "c_rk": 0.1, "max_depth": 30},
                    bg=bg, decide32=False)  # the FP64 definition, as the quadrature below
    ref = np.zeros((cam.h, cam.w, 4))
    for j in range(cam.h):
        for i in range(cam.w):
            org, d, amin, amax = O.pixel_ray(cam, i, j)
            ref[j, i] = BF.shell_ray_integral(f, tf, org, d, amin, amax, bg=bg)
    assert (fine["counts"] > 0).sum() > 10
    np.testing.assert_allclose(fine["rgba"], ref, atol=2e-7)


# ----------------------------------------------------------------- gradient --
def _loss(forest, tf, cam, integ, W, bg):
    r = O.render(forest, tf, cam, integ, bg=bg)
    return float((r["rgba"] * W).sum()), r["steps"]


@pytest.mark.parametrize("integ", [{"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16},
                                   {"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
                                   {"method": "simpson", "c_rk": 0.2, "max_depth": 16}])
@pytest.mark.parametrize("part", ["knots", "nodal"])
def test_shell_gradient_matches_central_differences(part, integ):
    """Reverse-mode gradient on the shell (27 nodal values per leaf) against
    central differences of the forward oracle, as for the cube."""
    f, tf = _shell(1, 1)
    if part == "nodal":
        k = np.arange(8)
        tf.knots[:] = np.column_stack([0.5 + k, 0.1 + 0.1 * k, 0.8 - 0.1 * k, 0.3 + 0.05 * k])
        span = float(f.nodal.max() - f.nodal.min())
        tf.s_min, tf.s_max = float(f.nodal.min()) - 0.5 * span, float(f.nodal.max()) + 0.5 * span
    cam = I.perspective_camera(5, 8, 6, dist=(2.0, 2.4), target=(0.0, 0.0, 0.0))
    bg = (0.2, 0.1, 0.05)
    rng = np.random.default_rng(13)
    W = rng.uniform(-1, 1, (cam.h, cam.w, 4))
    gn, gt = O.render_grad(f, tf, cam, integ, W, bg=bg)
    assert gn.shape == (f.nleaves, 27) and np.abs(gn).max() > 0 and np.abs(gt).max() > 0
    if part == "knots":
        coords, arr, g = range(32), tf.knots.reshape(-1), gt.reshape(-1)
    else:
        hot = np.flatnonzero(np.abs(gn).reshape(-1) > 1e-3 * np.abs(gn).max())
        coords, arr, g = rng.choice(hot, 24, replace=False), f.nodal.reshape(-1), gn.reshape(-1)
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
    assert checked >= (24 if part == "knots" else 20)  # the rest changed the step tree


# ------------------------------------------------------------------ surfaces --
def _radial_shell(level):
    """A uniform shell whose nodal values are the normalised radius zeta
    (exactly representable by the degree-2 data): the isosurfaces of the
    field are the spheres |x| = r0 + zeta (r1 - r0)."""
    f, tf = _shell(level, level)
    r0, r1 = f.meta["r0"], f.meta["r1"]
    L = f.max_level
    for k in range(f.nleaves):
        z0 = f.anchor[k, 2] * 2.0 ** -L
        h = 2.0 ** -int(f.level[k])
        for c in range(27):
            f.nodal[k, c] = np.float32(z0 + h * (c // 9) / 2.0)
    return f, tf, r0, r1


def test_shell_field_gradient_matches_central_differences():
    """The field's spatial gradient (the surface normal of Sec. 2.8) through
    the inverse map and the degree-2 basis, against central differences of
    the field in space at points inside leaves of a noise-field shell."""
    f, tf = _shell(1, 2)
    of = O.OracleForest(f, tf)
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(200):
        leaf = int(rng.integers(f.nleaves))
        L = f.max_level
        h = 2.0 ** -int(f.level[leaf])
        ref = f.anchor[leaf] * 2.0 ** -L + h * rng.uniform(0.2, 0.8, 3)
        x = np.asarray(O.shell_map(of, int(f.tree[leaf]), ref))
        d = np.array([0.3, -0.2, 0.9])
        s, g = O.field_probe(of, leaf, x, d, 0.0, 0.0)
        fd = np.zeros(3)
        e = 1e-6
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a] += e
            xm[a] -= e
            fd[a] = (O.field_probe(of, leaf, xp, d, 0.0, 0.0)[0] -
                     O.field_probe(of, leaf, xm, d, 0.0, 0.0)[0]) / (2 * e)
        assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), (leaf, g, fd)
        checked += 1
    assert checked == 200


def test_shell_isosurface_segment_closed_form():
    """Sec. 2.8 on the shell: with the field equal to the normalised radius
    and a constant medium, a ray through one leaf that crosses the sphere
    |x| = R_iso (s_iso = 1/2) gives near volume (+) surface (+) far volume in
    closed form: each volume piece exp(-kappa L), q (1 - A) / kappa over its
    chord, the surface A = a_s^(1/cos phi), B = i_s (1 - A) with phi the angle
    between the ray and the radial normal at the crossing (Eqs. 2.18, 2.35)."""
    f, tf, r0, r1 = _radial_shell(0)
    kap, q = 2.5, np.array([0.3, 0.6, 0.9], np.float32).astype(float)  # the knots are float32
    tf.knots[:] = np.concatenate([[kap], q])
    tf.s_min, tf.s_max = -1.0, 2.0
    of = O.OracleForest(f, tf)
    integ = {"method": "dopri5", "tol": 1e-12, "c_rk": 0.05, "max_depth": 30,
             "surface": {"s_iso": 0.5, "a_s": 0.6, "i_s": (1.0, 0.5, 0.25)}}
    R = r0 + 0.5 * (r1 - r0)
    org = np.array([2.0, 0.05, 0.1])
    d = np.array([-1.0, 0.02, -0.03])  # enters tree +x through the outer sphere
    hits = [(leaf, iv) for leaf in range(f.nleaves)
            for iv in O.ray_leaf_intervals(of, leaf, org, d, 0.0, 1e9)[0]]
    leaf, (a_in, a_out) = next((l, iv) for l, iv in hits
                               if np.linalg.norm(org + iv[0] * d) > R > np.linalg.norm(org + iv[1] * d)
                               or np.linalg.norm(org + iv[1] * d) > R > np.linalg.norm(org + iv[0] * d))
    seg, _ = O.segment_ab(of, integ, leaf, org, d, a_in, a_out)
    # crossing of |o + a d| = R inside [a_in, a_out]
    b, c = org @ d / (d @ d), (org @ org - R * R) / (d @ d)
    roots = [-b - math.sqrt(b * b - c), -b + math.sqrt(b * b - c)]
    ac = next(a for a in roots if a_in < a < a_out)
    xc = org + ac * d
    cphi = abs(xc @ d) / (np.linalg.norm(xc) * np.linalg.norm(d))
    rl = np.linalg.norm(d)

    def piece(L):
        A = math.exp(-kap * L)
        return np.array([A, *(q * (1 - A) / kap)])

    def comb(n, fa):  # Eq. 2.14, n nearer
        return np.array([n[0] * fa[0], *(n[1:] + n[0] * fa[1:])])
    As = 0.6 ** (1.0 / cphi)
    surf = np.array([As, *(np.array([1.0, 0.5, 0.25]) * (1 - As))])
    exp = comb(piece((ac - a_in) * rl), comb(surf, piece((a_out - ac) * rl)))
    np.testing.assert_allclose(seg, exp, rtol=1e-9, atol=1e-12)
