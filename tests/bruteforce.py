"""Brute-force references used to pin the oracle (test helpers, NumPy only).

None of these use leaves as segments, the segment group action, or the
oracle's code: they evaluate the defining integrals directly.

* ``ray_integral``: Eq. 2.12 of the paper along a whole ray,
  A = exp(-int kappa), B = int q(x) exp(-int_x^{x2} kappa), by the composite
  trapezoid rule on a fine grid, with the medium found by point location.
* ``leaves_along_ray``: the leaves a ray passes, found by point location at
  the midpoints between consecutive crossings of finest-level grid planes.
"""
from __future__ import annotations

import numpy as np


def tf_numpy(tf, s):
    """Piecewise-linear transfer function via np.interp (clamped outside)."""
    xs = tf.s_min + np.arange(8) * (tf.s_max - tf.s_min) / 7.0
    k = tf.knots.astype(np.float64)
    return np.stack([np.interp(s, xs, k[:, c]) for c in range(4)], axis=-1)


def locate(forest, pts):
    """Index of the leaf containing each point (unit cube; -1 outside)."""
    L = forest.max_level
    n = 1 << L
    pts = np.asarray(pts)
    q = np.floor(pts * n).astype(np.int64)
    # the cube is closed: points on its faces (up to rounding) belong to it
    inside = np.all((pts >= -1e-12) & (pts <= 1.0 + 1e-12), axis=-1)
    q = np.clip(q, 0, n - 1)
    # dense lookup table at the finest level (small meshes only)
    if not hasattr(forest, "_lut"):
        lut = -np.ones((n, n, n), dtype=np.int64)
        for idx in range(forest.nleaves):
            a = forest.anchor[idx]
            sz = 1 << (L - int(forest.level[idx]))
            lut[a[0]:a[0] + sz, a[1]:a[1] + sz, a[2]:a[2] + sz] = idx
        forest._lut = lut
    out = forest._lut[q[..., 0], q[..., 1], q[..., 2]]
    return np.where(inside, out, -1)


def field_at(forest, pts):
    """Trilinear field value at points via scipy's RegularGridInterpolator per leaf."""
    pts = np.asarray(pts, dtype=np.float64)
    leaf = locate(forest, pts)
    out = np.zeros(pts.shape[:-1])
    L = forest.max_level
    for idx in np.unique(leaf[leaf >= 0]):
        m = leaf == idx
        a = forest.anchor[idx] / float(1 << L)
        h = 2.0 ** -int(forest.level[idx])
        u = (pts[m] - a) / h
        v = forest.nodal[idx].astype(np.float64).reshape(2, 2, 2)  # [bz, by, bx]
        from scipy.interpolate import RegularGridInterpolator
        rgi = RegularGridInterpolator(([0.0, 1.0], [0.0, 1.0], [0.0, 1.0]), v.transpose(2, 1, 0),
                                      bounds_error=False, fill_value=None)
        out[m] = rgi(u)
    return out, leaf


def chord(org, d, amin, amax):
    """Parameter interval of the ray inside the unit cube (clipped to [amin, amax])."""
    t0, t1 = amin, amax
    for a in range(3):
        if d[a] == 0.0:
            if not (0.0 <= org[a] <= 1.0):
                return None
            continue
        s0, s1 = sorted(((0.0 - org[a]) / d[a], (1.0 - org[a]) / d[a]))
        t0, t1 = max(t0, s0), min(t1, s1)
    return (t0, t1) if t1 > t0 else None


def ray_integral(forest, tf, org, d, amin, amax, npts=200001, bg=(0.0, 0.0, 0.0)):
    """(r, g, b, alpha) of one ray by quadrature of the closed-form solution."""
    ch = chord(org, d, amin, amax)
    if ch is None:
        return np.array([bg[0], bg[1], bg[2], 0.0])
    a0, a1 = ch
    rl = float(np.linalg.norm(d))
    # x = world distance from the far end; alpha(x) = a1 - x / |r|
    xs = np.linspace(0.0, (a1 - a0) * rl, npts)
    pts = org[None, :] + (a1 - xs / rl)[:, None] * d[None, :]
    s, leaf = field_at(forest, pts)
    kq = tf_numpy(tf, s)
    kq[leaf < 0] = 0.0
    kap, q = kq[:, 0], kq[:, 1:]
    dx = xs[1] - xs[0]
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * dx)])  # int_0^x kappa
    A = np.exp(-tau[-1])
    wgt = np.exp(-(tau[-1] - tau))  # exp(-int_x^{x2} kappa)
    f = q * wgt[:, None]
    B = (0.5 * (f[1:] + f[:-1]) * dx).sum(axis=0)
    I = A * np.asarray(bg) + B
    return np.array([I[0], I[1], I[2], 1.0 - A])


def leaves_along_ray(forest, org, d, amin, amax):
    """Ordered list of leaves a ray passes (consecutive duplicates merged)."""
    ch = chord(org, d, amin, amax)
    if ch is None:
        return []
    a0, a1 = ch
    n = 1 << forest.max_level
    cuts = [a0, a1]
    for a in range(3):
        if d[a] != 0.0:
            ks = np.arange(1, n)
            al = (ks / n - org[a]) / d[a]
            cuts.extend(al[(al > a0) & (al < a1)].tolist())
    cuts = np.unique(np.asarray(cuts))
    mids = 0.5 * (cuts[1:] + cuts[:-1])
    pts = org[None, :] + mids[:, None] * d[None, :]
    leaf = locate(forest, pts)
    out = []
    for l in leaf:
        if l >= 0 and (not out or out[-1] != l):
            out.append(int(l))
    return out


# ------------------------------------------------------------ shell forests --
# Point location in a cubed-sphere shell, written from the definition of the
# equiangular map: the tree of a point is the cube face its central projection
# lands on (the largest x . n over the six face normals); its reference
# coordinates invert the map.

def shell_ref(forest, pts):
    """Tree and reference coordinates (xi, eta, zeta) of points [..., 3]."""
    fr = np.asarray(forest.meta["frames"], dtype=np.float64)
    r0, r1 = forest.meta["r0"], forest.meta["r1"]
    pts = np.asarray(pts, dtype=np.float64)
    tree = np.argmax(pts @ fr[:, 0, :].T, axis=-1)
    f = fr[tree]
    pn = np.einsum("...i,...i->...", pts, f[..., 0, :])
    xi = np.arctan(np.einsum("...i,...i->...", pts, f[..., 1, :]) / pn) / (np.pi / 2) + 0.5
    eta = np.arctan(np.einsum("...i,...i->...", pts, f[..., 2, :]) / pn) / (np.pi / 2) + 0.5
    zeta = (np.linalg.norm(pts, axis=-1) - r0) / (r1 - r0)
    return tree, np.stack([xi, eta, zeta], axis=-1)


def shell_locate(forest, pts, clip_radial=False):
    """Leaf containing each point (-1 in the hollow or outside) and the
    point's local coordinates in that leaf."""
    L = forest.max_level
    n = 1 << L
    tree, ref = shell_ref(forest, pts)
    if clip_radial:
        ref[..., 2] = np.clip(ref[..., 2], 0.0, 1.0)
    if not hasattr(forest, "_shell_lut"):
        lut = -np.ones((6, n, n, n), dtype=np.int64)
        for idx in range(forest.nleaves):
            a = forest.anchor[idx]
            sz = 1 << (L - int(forest.level[idx]))
            lut[forest.tree[idx], a[0]:a[0] + sz, a[1]:a[1] + sz, a[2]:a[2] + sz] = idx
        forest._shell_lut = lut
    inside = (ref[..., 2] >= -1e-12) & (ref[..., 2] <= 1.0 + 1e-12)
    q = np.clip(np.floor(ref * n).astype(np.int64), 0, n - 1)
    leaf = np.where(inside, forest._shell_lut[tree, q[..., 0], q[..., 1], q[..., 2]], -1)
    lv = forest.level[np.maximum(leaf, 0)].astype(np.float64)
    h = 2.0 ** -lv
    u = (ref - forest.anchor[np.maximum(leaf, 0)] / float(n)) / h[..., None]
    return leaf, u


def shell_field_at(forest, pts, clip_radial=False):
    """Degree-2 Lagrange interpolation on {0, 1/2, 1}^3 of the 27 nodal values."""
    leaf, u = shell_locate(forest, pts, clip_radial)

    def basis(t):  # [..., 3]: the three quadratic Lagrange polynomials
        return np.stack([(t - 0.5) * (t - 1.0) / 0.5, -t * (t - 1.0) / 0.25,
                         t * (t - 0.5) / 0.5], axis=-1)

    bu, bv, bw = basis(u[..., 0]), basis(u[..., 1]), basis(u[..., 2])
    w = np.einsum("...a,...b,...c->...cba", bu, bv, bw).reshape(u.shape[:-1] + (27,))
    vals = forest.nodal[np.maximum(leaf, 0)].astype(np.float64)
    return (vals * w).sum(axis=-1), leaf


def ball_interval(org, d, r):
    """Parameter interval of the ray inside the ball |x| <= r (None if missed)."""
    a, b, c = d @ d, org @ d, org @ org - r * r
    disc = b * b - a * c
    if disc <= 0.0:
        return None
    s = np.sqrt(disc)
    return (-b - s) / a, (-b + s) / a


def shell_pieces(forest, org, d, amin, amax):
    """The ray's intervals inside the shell r0 <= |x| <= r1, nearest first."""
    outer = ball_interval(org, d, forest.meta["r1"])
    if outer is None:
        return []
    t0, t1 = max(amin, outer[0]), min(amax, outer[1])
    inner = ball_interval(org, d, forest.meta["r0"])
    pieces = [(t0, t1)] if inner is None else [(t0, min(t1, inner[0])), (max(t0, inner[1]), t1)]
    return [p for p in pieces if p[1] > p[0]]


def _quad_piece(values_at, org, d, a0, a1, npts, tf):
    rl = float(np.linalg.norm(d))
    xs = np.linspace(0.0, (a1 - a0) * rl, npts)
    pts = org[None, :] + (a1 - xs / rl)[:, None] * d[None, :]
    s, leaf = values_at(pts)
    kq = tf_numpy(tf, s)
    kq[leaf < 0] = 0.0
    kap, q = kq[:, 0], kq[:, 1:]
    dx = xs[1] - xs[0]
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * dx)])
    wgt = np.exp(-(tau[-1] - tau))
    f = q * wgt[:, None]
    return np.exp(-tau[-1]), (0.5 * (f[1:] + f[:-1]) * dx).sum(axis=0)


def shell_ray_integral(forest, tf, org, d, amin, amax, npts=100001, bg=(0.0, 0.0, 0.0)):
    """(r, g, b, alpha) of one ray through a shell by quadrature of the closed
    form on each piece of the ray inside the shell, the pieces applied to the
    intensity far to near (Eq. 2.11)."""
    I, T = np.asarray(bg, dtype=np.float64), 1.0
    for a0, a1 in reversed(shell_pieces(forest, org, d, amin, amax)):
        A, B = _quad_piece(lambda p: shell_field_at(forest, p, clip_radial=True), org, d, a0, a1,
                           npts, tf)
        I = A * I + B
        T *= A
    return np.array([I[0], I[1], I[2], 1.0 - T])


def shell_leaves_along_ray(forest, org, d, amin, amax):
    """Leaves a ray passes in a shell, near to far, a leaf entered twice (across
    the hollow) listed twice: point location at the midpoints between all
    crossings of the finest level's boundary planes (through the origin) and
    spheres."""
    fr = np.asarray(forest.meta["frames"], dtype=np.float64)
    r0, r1 = forest.meta["r0"], forest.meta["r1"]
    n = 1 << forest.max_level
    cuts = [amin, amax]
    for r in r0 + (r1 - r0) * np.arange(n + 1) / n:
        iv = ball_interval(org, d, r)
        if iv is not None:
            cuts.extend(iv)
    tk = np.tan(np.pi / 4 * (2 * np.arange(n + 1) / n - 1))
    for t in range(6):
        for e in (fr[t, 1], fr[t, 2]):
            m = e[None, :] - tk[:, None] * fr[t, 0][None, :]
            g1 = m @ d
            ok = g1 != 0.0
            cuts.extend((-(m[ok] @ org) / g1[ok]).tolist())
    cuts = np.unique(np.asarray(cuts))
    cuts = cuts[(cuts >= amin) & (cuts <= amax)]
    mids = 0.5 * (cuts[1:] + cuts[:-1])
    leaf, _ = shell_locate(forest, org[None, :] + mids[:, None] * d[None, :])
    out, prev = [], -1
    for l in leaf:
        if l >= 0 and l != prev:
            out.append(int(l))
        prev = l
    return out
