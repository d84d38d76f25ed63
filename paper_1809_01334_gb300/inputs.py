"""Seeded synthetic inputs for the forest-of-octrees raycaster.

This module builds the *inputs* of the raycaster: the linear forest of octree
leaves (the domain description of Sec. 2.1), the per-leaf nodal field values,
the piecewise-linear transfer function and the cameras (Sec. 2.2).  Both the
FP64 oracle and the CUDA path read what it produces, so it holds none of the
raycasting arithmetic: no camera transform, no bounding boxes, no ray/leaf
intersection, no integration and no segment algebra.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that the
inputs are bit-identical on every machine and NumPy version.

Layout of a forest (all host NumPy arrays):

* ``level``  uint8  [N]      refinement level of each leaf (root = 0)
* ``anchor`` int32  [N, 3]   lower corner of the leaf in integer units of
  ``2**-max_level`` of its tree's reference cube
* ``tree``   int32  [N]      tree index (0 for the single-tree unit cube)
* ``nodal``  float32 [N, 8]  field values at the leaf's 8 corners; corner
  ``c = bx + 2*by + 4*bz`` sits at ``anchor + (bx, by, bz) * size``

Leaves are sorted by (tree, Morton key of the anchor): the space-filling-curve
order of Sec. 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SplitMix64", "GaussianField", "Forest", "TransferFunction", "Camera",
    "gaussian_field", "uniform_cube_forest", "adaptive_cube_forest",
    "transfer_function", "ortho_camera_c1", "perspective_camera", "morton_keys",
    "preset_c1", "preset_c2", "preset_c4", "preset_small", "batch_cameras",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


class SplitMix64:
    """Counter-based SplitMix64 stream: the k-th draw depends only on (seed, k)."""

    GAMMA = np.uint64(0x9E3779B97F4A7C15)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def next_u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.state + self.GAMMA * k
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# Synthetic scalar field: a sum of isotropic Gaussians with unit amplitude.
# --------------------------------------------------------------------------
@dataclass
class GaussianField:
    centres: np.ndarray  # [K, 3]
    widths: np.ndarray   # [K]

    def value(self, pts: np.ndarray) -> np.ndarray:
        pts = np.asarray(pts, dtype=np.float64)
        out = np.zeros(pts.shape[:-1], dtype=np.float64)
        for c, s in zip(self.centres, self.widths):
            d2 = ((pts - c) ** 2).sum(axis=-1)
            out += np.exp(-d2 / (2.0 * s * s))
        return out

    def grad_norm(self, pts: np.ndarray) -> np.ndarray:
        pts = np.asarray(pts, dtype=np.float64)
        g = np.zeros(pts.shape, dtype=np.float64)
        for c, s in zip(self.centres, self.widths):
            d = pts - c
            e = np.exp(-(d * d).sum(axis=-1) / (2.0 * s * s)) / (s * s)
            g -= d * e[..., None]
        return np.sqrt((g * g).sum(axis=-1))


def gaussian_field(n_gauss: int, seed: int) -> GaussianField:
    """Centres uniform in [0.2, 0.8]^3, widths uniform in [0.05, 0.2]."""
    rng = SplitMix64(seed)
    u = rng.uniform(4 * n_gauss).reshape(n_gauss, 4)
    centres = 0.2 + 0.6 * u[:, :3]
    widths = 0.05 + 0.15 * u[:, 3]
    return GaussianField(centres, widths)


# --------------------------------------------------------------------------
# Forest
# --------------------------------------------------------------------------
def _part1by2(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_keys(anchor: np.ndarray) -> np.ndarray:
    """Interleave the bits of (x, y, z) anchors, x in the lowest bit."""
    a = np.asarray(anchor)
    return _part1by2(a[:, 0]) | (_part1by2(a[:, 1]) << np.uint64(1)) | (_part1by2(a[:, 2]) << np.uint64(2))


@dataclass
class Forest:
    geometry: str
    max_level: int
    level: np.ndarray
    anchor: np.ndarray
    tree: np.ndarray
    nodal: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nleaves(self) -> int:
        return int(self.level.shape[0])

    def leaf_boxes(self) -> tuple[np.ndarray, np.ndarray]:
        """World-space lower corner and edge length of each leaf (unit cube, identity map)."""
        scale = 2.0 ** -self.max_level
        size = (2.0 ** (self.max_level - self.level.astype(np.float64))) * scale
        return self.anchor.astype(np.float64) * scale, size


def _sort_forest(level, anchor, tree):
    key = morton_keys(anchor)
    order = np.lexsort((key, tree))
    return level[order], anchor[order], tree[order]


def _axis_tables(fld: GaussianField, n: int):
    """Per-Gaussian, per-axis factors on the grid k / n, k = 0..n (the Gaussians are separable)."""
    x = np.arange(n + 1, dtype=np.float64) / n
    inv = 1.0 / (2.0 * fld.widths ** 2)
    e = [np.exp(-((x[None, :] - fld.centres[:, a, None]) ** 2) * inv[:, None]) for a in range(3)]
    de = [-(x[None, :] - fld.centres[:, a, None]) / (fld.widths[:, None] ** 2) * e[a] for a in range(3)]
    return e, de


def _sample_corners(fld: GaussianField, level, anchor, max_level, chunk=1 << 19):
    """Field values at the 8 corners of every leaf, in FP64, stored as float32."""
    n = level.shape[0]
    out = np.empty((n, 8), dtype=np.float32)
    (ex, ey, ez), _ = _axis_tables(fld, 1 << max_level)
    size = (1 << (max_level - level.astype(np.int64)))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        a = anchor[s:e].astype(np.int64)
        sz = size[s:e]
        for c in range(8):
            ix = a[:, 0] + (c & 1) * sz
            iy = a[:, 1] + ((c >> 1) & 1) * sz
            iz = a[:, 2] + ((c >> 2) & 1) * sz
            out[s:e, c] = (ex[:, ix] * ey[:, iy] * ez[:, iz]).sum(axis=0).astype(np.float32)
    return out


def _grad_norm_grid(fld: GaussianField, n: int, centres: bool) -> np.ndarray:
    """|grad f| on the (n+1)^3 vertex grid of level log2(n), or on its n^3 cell centres."""
    if centres:
        x = (np.arange(n, dtype=np.float64) + 0.5) / n
        inv = 1.0 / (2.0 * fld.widths ** 2)
        e = [np.exp(-((x[None, :] - fld.centres[:, a, None]) ** 2) * inv[:, None]) for a in range(3)]
        de = [-(x[None, :] - fld.centres[:, a, None]) / (fld.widths[:, None] ** 2) * e[a] for a in range(3)]
    else:
        e, de = _axis_tables(fld, n)
    m = e[0].shape[1]
    g = np.zeros((3, m, m, m))
    for k in range(fld.widths.shape[0]):
        g[0] += de[0][k][:, None, None] * e[1][k][None, :, None] * e[2][k][None, None, :]
        g[1] += e[0][k][:, None, None] * de[1][k][None, :, None] * e[2][k][None, None, :]
        g[2] += e[0][k][:, None, None] * e[1][k][None, :, None] * de[2][k][None, None, :]
    return np.sqrt((g * g).sum(axis=0))


def uniform_cube_forest(level: int, fld: GaussianField, max_level: int | None = None) -> Forest:
    """Unit cube uniformly refined to ``level`` (8**level leaves), Morton order."""
    L = level if max_level is None else max_level
    n1 = 1 << level
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij"), -1).reshape(-1, 3)
    anchor = (g << (L - level)).astype(np.int32)
    lev = np.full(anchor.shape[0], level, dtype=np.uint8)
    tree = np.zeros(anchor.shape[0], dtype=np.int32)
    lev, anchor, tree = _sort_forest(lev, anchor, tree)
    nodal = _sample_corners(fld, lev, anchor, L)
    return Forest("cube", L, lev, anchor, tree, nodal, {"kind": "uniform", "level": level})


def _dilate26(a: np.ndarray) -> np.ndarray:
    p = np.pad(a, 1)
    out = np.zeros_like(a)
    n = a.shape[0]
    for dx in range(3):
        for dy in range(3):
            for dz in range(3):
                out |= p[dx:dx + n, dy:dy + n, dz:dz + n]
    return out


def _upsample(a: np.ndarray) -> np.ndarray:
    return a.repeat(2, 0).repeat(2, 1).repeat(2, 2)


def adaptive_cube_forest(fld: GaussianField, min_level: int, max_level: int, theta: float,
                         balance: bool = True) -> Forest:
    """Unit cube refined from ``min_level`` while h * max|grad f| > theta.

    ``max|grad f|`` is taken over a node's 8 corners and its centre; ``h`` is
    its edge length.  With ``balance`` the mesh is made 2:1 balanced across
    faces, edges and corners (the 26-neighbourhood).
    """
    refined = [np.zeros((1 << l,) * 3, dtype=bool) for l in range(max_level)]
    for l in range(min_level):
        refined[l][...] = True
    for l in range(min_level, max_level):
        n1 = 1 << l
        exists = np.ones((n1,) * 3, bool) if l == 0 else _upsample(refined[l - 1])
        h = 1.0 / n1
        gv = _grad_norm_grid(fld, n1, centres=False)
        gmax = _grad_norm_grid(fld, n1, centres=True)
        for dx in range(2):
            for dy in range(2):
                for dz in range(2):
                    np.maximum(gmax, gv[dx:dx + n1, dy:dy + n1, dz:dz + n1], out=gmax)
        refined[l] = exists & (h * gmax > theta)
    if balance:
        for l in range(max_level - 1, 0, -1):
            need = _dilate26(refined[l])
            m = 1 << (l - 1)
            refined[l - 1] |= need.reshape(m, 2, m, 2, m, 2).any(axis=(1, 3, 5))
    levs, anchors = [], []
    for l in range(0, max_level + 1):
        n1 = 1 << l
        exists = np.ones((n1,) * 3, bool) if l == 0 else _upsample(refined[l - 1])
        leaf = exists & ~refined[l] if l < max_level else exists
        idx = np.argwhere(leaf)
        if idx.shape[0]:
            anchors.append((idx << (max_level - l)).astype(np.int32))
            levs.append(np.full(idx.shape[0], l, dtype=np.uint8))
    lev = np.concatenate(levs)
    anchor = np.concatenate(anchors)
    tree = np.zeros(lev.shape[0], dtype=np.int32)
    lev, anchor, tree = _sort_forest(lev, anchor, tree)
    nodal = _sample_corners(fld, lev, anchor, max_level)
    return Forest("cube", max_level, lev, anchor, tree, nodal,
                  {"kind": "adaptive", "min_level": min_level, "max_level": max_level,
                   "theta": theta, "balanced": balance})


# --------------------------------------------------------------------------
# Transfer function: 8 knots, uniformly spaced over [s_min, s_max].
# --------------------------------------------------------------------------
@dataclass
class TransferFunction:
    knots: np.ndarray  # float32 [8, 4]: kappa, q_r, q_g, q_b at each knot
    s_min: float
    s_max: float

    def flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.knots, dtype=np.float32).reshape(-1)


def transfer_function(nodal: np.ndarray, seed: int = 1334, kappa_max: float = 20.0) -> TransferFunction:
    """Knot values kappa ~ U[0, kappa_max], q ~ U[0, 1]^3; range = min/max of the nodal data."""
    rng = SplitMix64(seed)
    u = rng.uniform(32).reshape(8, 4)
    knots = np.empty((8, 4), dtype=np.float32)
    knots[:, 0] = (kappa_max * u[:, 0]).astype(np.float32)
    knots[:, 1:] = u[:, 1:].astype(np.float32)
    s_min = float(np.float32(nodal.min()))
    s_max = float(np.float32(nodal.max()))
    if not s_max > s_min:
        s_max = float(np.float32(s_min + 1.0))
    return TransferFunction(knots, s_min, s_max)


# --------------------------------------------------------------------------
# Cameras (pinhole, Sec. 2.2; plus an orthographic variant).  Every number is
# rounded to float32 so that the FP32 and FP64 paths read identical constants.
# --------------------------------------------------------------------------
@dataclass
class Camera:
    o: tuple
    v: tuple
    t: tuple
    u: tuple
    ell: float
    near: float
    far: float
    w: int
    h: int
    ortho: bool = False


def _f32(x):
    return tuple(float(np.float32(c)) for c in x)


def ortho_camera_c1(w: int = 64, h: int = 64) -> Camera:
    """Looks down -z from z = 3 at the unit cube; the image tiles [0, 1]^2."""
    return Camera(o=(0.5, 0.5, 3.0), v=(0.0, 0.0, -1.0), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                  ell=float(np.float32(1.0 / max(w, h))), near=1.0, far=1e30, w=w, h=h, ortho=True)


def perspective_camera(seed: int, w: int, h: int, dist=(2.5, 3.5), fov_deg: float = 45.0,
                       near: float = 0.1, far: float = 100.0, target=(0.5, 0.5, 0.5)) -> Camera:
    """Camera at a seeded distance and uniform direction around ``target``, looking at it."""
    rng = SplitMix64(seed)
    a, b, c = rng.uniform(3)
    d = dist[0] + (dist[1] - dist[0]) * a
    z = 2.0 * b - 1.0
    phi = 2.0 * math.pi * c
    rxy = math.sqrt(max(0.0, 1.0 - z * z))
    direction = np.array([rxy * math.cos(phi), rxy * math.sin(phi), z])
    tgt = np.asarray(target, dtype=np.float64)
    o = tgt + d * direction
    fwd = -direction
    up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
    tv = np.cross(fwd, up)
    tv /= np.linalg.norm(tv)
    uv = np.cross(tv, fwd)
    ell = 2.0 * near * math.tan(math.radians(fov_deg) / 2.0) / h
    return Camera(o=_f32(o), v=_f32(near * fwd), t=_f32(tv), u=_f32(uv), ell=float(np.float32(ell)),
                  near=float(np.float32(near)), far=float(np.float32(far)), w=w, h=h, ortho=False)


# --------------------------------------------------------------------------
# Presets (forest/field seed 1809, transfer-function seed 1334, camera seed 7)
# --------------------------------------------------------------------------
C2_THETA = 0.0875  # calibrated once (bisection) to give 2,053,451 balanced leaves


def preset_c1():
    """Uniform level 3 (512 leaves), 4 Gaussians, orthographic 64x64, RK4 x 4 steps."""
    fld = gaussian_field(4, 1809)
    forest = uniform_cube_forest(3, fld)
    tf = transfer_function(forest.nodal, 1334)
    cam = ortho_camera_c1(64, 64)
    integ = {"method": "rk4", "nsteps": 4}
    return forest, tf, cam, integ


def preset_c2(w: int = 1920, h: int = 1080, theta: float = C2_THETA, max_level: int = 8):
    """Adaptive levels 2..8, 16 Gaussians, 2:1 balanced, perspective 45 deg, DOPRI5 tol 1e-6."""
    fld = gaussian_field(16, 1809)
    forest = adaptive_cube_forest(fld, 2, max_level, theta, balance=True)
    tf = transfer_function(forest.nodal, 1334)
    cam = perspective_camera(7, w, h)
    integ = {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}
    return forest, tf, cam, integ


def batch_cameras(n: int = 64, seed: int = 7, lo: int = 256, ratio: float = 8.0):
    """n square perspective cameras with sides round(lo * ratio**u), u ~ U[0, 1]
    (log-uniform sizes), each at its own seeded position."""
    rng = SplitMix64(seed)
    u = rng.uniform(n)
    return [perspective_camera(seed * 1000 + k, int(round(lo * ratio ** u[k])),
                               int(round(lo * ratio ** u[k]))) for k in range(n)]


def preset_c4(n: int = 64):
    """The C2 forest, field and transfer function seen by n cameras of
    log-uniform sizes 256^2 .. 2048^2."""
    forest, tf, _, integ = preset_c2()
    return forest, tf, batch_cameras(n), integ


def preset_small(kind: str = "adaptive", seed: int = 1809, w: int = 48, h: int = 40,
                 theta: float = 0.25, max_level: int = 4, cam_seed: int = 7):
    """Small cases the oracle finishes in seconds: still many tiles and a ragged image edge."""
    fld = gaussian_field(16 if kind == "adaptive" else 4, seed)
    if kind == "adaptive":
        forest = adaptive_cube_forest(fld, 1, max_level, theta, balance=True)
    else:
        forest = uniform_cube_forest(int(kind[-1]) if kind.startswith("uniform") else 2, fld)
    tf = transfer_function(forest.nodal, 1334)
    cam = perspective_camera(cam_seed, w, h)
    return forest, tf, cam


# --------------------------------------------------------------------------
# Cubed-sphere shell: six trees, the equiangular map, degree-2 nodal data.
# --------------------------------------------------------------------------
SHELL_R0, SHELL_R1 = 0.55, 1.0

# tree k: (face normal, first tangent, second tangent); reference coordinates
# (xi, eta, zeta) map to r(zeta) * normalize(n + tan(pi/4 (2 xi - 1)) e1 +
# tan(pi/4 (2 eta - 1)) e2), r(zeta) = R0 + (R1 - R0) zeta
SHELL_FRAMES = np.array([
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    [[-1, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 1, 0], [0, 0, 1], [1, 0, 0]],
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
    [[0, 0, 1], [1, 0, 0], [0, 1, 0]],
    [[0, 0, -1], [0, 1, 0], [1, 0, 0]]], dtype=np.float64)


def shell_map(tree, xi, eta, zeta):
    """Equiangular cubed-sphere map of tree reference coordinates to space."""
    fr = SHELL_FRAMES[np.asarray(tree)]
    a = np.tan(np.pi / 4 * (2 * np.asarray(xi) - 1))[..., None]
    b = np.tan(np.pi / 4 * (2 * np.asarray(eta) - 1))[..., None]
    d = fr[..., 0, :] + a * fr[..., 1, :] + b * fr[..., 2, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return (SHELL_R0 + (SHELL_R1 - SHELL_R0) * np.asarray(zeta))[..., None] * d


@dataclass
class ShellNoise:
    """f(x) = sum_{l<=lmax} sum_m c_lm Y_lm(x/|x|) (1 + sin(2 pi l zeta)/2),
    c_lm ~ N(0, 1/(l+1)), real spherical harmonics, zeta the normalised radius."""
    coef: dict
    lmax: int

    def direction_terms(self, d):
        """A_l(d) = sum_m c_lm Y_lm(d) for l = 0..lmax; d unit vectors [..., 3]."""
        ct = np.clip(d[..., 2], -1.0, 1.0)
        st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        phi = np.arctan2(d[..., 1], d[..., 0])
        out = np.zeros((self.lmax + 1,) + ct.shape)
        pmm = np.ones_like(ct)
        for m in range(self.lmax + 1):
            if m > 0:
                pmm = pmm * (2 * m - 1) * st
            pl2, pl1 = None, pmm
            for l in range(m, self.lmax + 1):
                if l == m:
                    p = pmm
                elif l == m + 1:
                    p = ct * (2 * m + 1) * pmm
                else:
                    p = ((2 * l - 1) * ct * pl1 - (l + m - 1) * pl2) / (l - m)
                if l > m:
                    pl2, pl1 = pl1, p
                k = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) /
                              math.factorial(l + m))
                if m == 0:
                    out[l] += self.coef[(l, 0)] * k * p
                else:
                    out[l] += math.sqrt(2.0) * k * p * (self.coef[(l, m)] * np.cos(m * phi) +
                                                        self.coef[(l, -m)] * np.sin(m * phi))
        return out

    @staticmethod
    def radial_terms(zeta, lmax):
        return np.stack([1.0 + 0.5 * np.sin(2 * np.pi * l * np.asarray(zeta))
                         for l in range(lmax + 1)])

    def value(self, pts):
        pts = np.asarray(pts, dtype=np.float64)
        r = np.linalg.norm(pts, axis=-1)
        A = self.direction_terms(pts / r[..., None])
        R = self.radial_terms((r - SHELL_R0) / (SHELL_R1 - SHELL_R0), self.lmax)
        return (A * R).sum(axis=0)


def shell_noise(seed: int = 1809, lmax: int = 8) -> ShellNoise:
    rng = SplitMix64(seed)
    coef = {}
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            u1, u2 = rng.uniform(2)
            g = math.sqrt(-2.0 * math.log(max(u1, 1e-300))) * math.cos(2 * math.pi * u2)
            coef[(l, m)] = g / math.sqrt(l + 1.0)
    return ShellNoise(coef, lmax)


def shell_forest(noise: ShellNoise, min_level: int, max_level: int, theta: float) -> Forest:
    """Six trees refined from min_level while the noise varies by more than
    theta over a node (its 8 corners and centre), not balanced.  Nodal data:
    27 values per leaf at the leaf's local nodes (a, b, c)/2, node index
    a + 3 b + 9 c (the degree-2 Gauss-Lobatto nodes 0, 1/2, 1)."""
    L = max_level
    n2 = 1 << (L + 1)                      # the finest node grid: level L + 1
    g = np.arange(n2 + 1) / n2
    XI, ETA = np.meshgrid(g, g, indexing="ij")
    A = np.empty((6, noise.lmax + 1, n2 + 1, n2 + 1))
    for t in range(6):
        d = shell_map(np.full(XI.shape, t), XI, ETA, np.zeros(XI.shape))
        A[t] = noise.direction_terms(d / np.linalg.norm(d, axis=-1, keepdims=True))
    R = ShellNoise.radial_terms(g, noise.lmax)  # [lmax + 1, n2 + 1]

    ls = np.arange(noise.lmax + 1)[None, :]

    def f_at(t, ix, iy, iz):  # f at points of the level-(L + 1) node grid
        return (A[t[:, None], ls, ix[:, None], iy[:, None]] * R[:, iz].T).sum(axis=1)

    levs, anchors, trees = [], [], []
    for t in range(6):
        refined = [np.zeros((1 << l,) * 3, bool) for l in range(L)]
        for l in range(min_level):
            refined[l][...] = True
        for l in range(min_level, L):
            n1 = 1 << l
            exists = np.ones((n1,) * 3, bool) if l == 0 else _upsample(refined[l - 1])
            idx = np.argwhere(exists)
            if idx.shape[0] == 0:
                continue
            step = 1 << (L + 1 - l)  # node-grid units per level-l cell
            vals = []
            for c in range(9):
                off = np.array([1, 1, 1]) if c == 8 else np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]) * 2
                p = idx * step + off * (step // 2)
                vals.append(f_at(np.full(idx.shape[0], t), p[:, 0], p[:, 1], p[:, 2]))
            vals = np.stack(vals)
            ref = (vals.max(axis=0) - vals.min(axis=0)) > theta
            refined[l][tuple(idx[ref].T)] = True
        for l in range(0, L + 1):
            n1 = 1 << l
            exists = np.ones((n1,) * 3, bool) if l == 0 else _upsample(refined[l - 1])
            leaf = exists & ~refined[l] if l < L else exists
            idx = np.argwhere(leaf)
            if idx.shape[0]:
                anchors.append((idx << (L - l)).astype(np.int32))
                levs.append(np.full(idx.shape[0], l, dtype=np.uint8))
                trees.append(np.full(idx.shape[0], t, dtype=np.int32))
    lev = np.concatenate(levs)
    anchor = np.concatenate(anchors)
    tree = np.concatenate(trees)
    lev, anchor, tree = _sort_forest(lev, anchor, tree)
    nodal = np.empty((lev.shape[0], 27), dtype=np.float32)
    step = (1 << (L + 1 - lev.astype(np.int64))) // 2  # node-grid units per half leaf
    for c in range(27):
        a, b, cc = c % 3, (c // 3) % 3, c // 9
        ix = 2 * anchor[:, 0].astype(np.int64) + a * step
        iy = 2 * anchor[:, 1].astype(np.int64) + b * step
        iz = 2 * anchor[:, 2].astype(np.int64) + cc * step
        nodal[:, c] = f_at(tree, ix, iy, iz).astype(np.float32)
    return Forest("shell", L, lev, anchor, tree, nodal,
                  {"kind": "shell", "min_level": min_level, "max_level": max_level,
                   "theta": theta, "r0": SHELL_R0, "r1": SHELL_R1,
                   "frames": SHELL_FRAMES.tolist()})


C3_THETA = 0.38  # calibrated once (bisection) to give 5,001,233 leaves over levels 4..7


def preset_c3(w: int = 2048, h: int = 2048, theta: float = C3_THETA, min_level: int = 4,
              max_level: int = 7):
    """Cubed-sphere shell, levels 4..7, degree-2 data from SH noise (degree 8),
    perspective 45 deg at 2048^2, DOPRI5 tol 1e-5."""
    noise = shell_noise(1809, 8)
    forest = shell_forest(noise, min_level, max_level, theta)
    tf = transfer_function(forest.nodal, 1334)
    cam = perspective_camera(7, w, h, target=(0.0, 0.0, 0.0))
    integ = {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16}
    return forest, tf, cam, integ


C5_THETA = 0.5  # calibrated once to give 1,082,535 leaves over levels 4..6


def preset_c5(w: int = 1024, h: int = 1024, theta: float = C5_THETA, min_level: int = 4,
              max_level: int = 6):
    """Cubed-sphere shell, levels 4..6, degree-2 data from SH noise (degree 8),
    perspective 45 deg at 1024^2, DOPRI5 tol 1e-5 (the differentiation
    workload; its target is rendered from a seeded 5% perturbation)."""
    noise = shell_noise(1809, 8)
    forest = shell_forest(noise, min_level, max_level, theta)
    tf = transfer_function(forest.nodal, 1334)
    cam = perspective_camera(7, w, h, target=(0.0, 0.0, 0.0))
    integ = {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16}
    return forest, tf, cam, integ


def preset_shell_small(w: int = 40, h: int = 32, min_level: int = 1, max_level: int = 3,
                       theta: float = 2.0, cam_seed: int = 7):
    noise = shell_noise(1809, 8)
    forest = shell_forest(noise, min_level, max_level, theta)
    tf = transfer_function(forest.nodal, 1334)
    cam = perspective_camera(cam_seed, w, h, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    return forest, tf, cam
