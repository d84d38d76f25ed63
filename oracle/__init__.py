"""FP64 CPU oracle for the forest-of-octrees raycaster (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_1809_01334_gb300/csrc``; the two meet
only in the seeded inputs of ``paper_1809_01334_gb300.inputs``, which hold no
raycasting arithmetic.

The C source (``ocr_oracle.c``) states, function by function, which equation
or algorithm of the paper it writes out.  Every function is pinned by
``tests/test_oracle_pins.py`` to closed forms, invariants or brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libocr_oracle.so")
_lib = None

RK4, DOPRI5, GAUSS2, SIMPSON, EQUILIBRIUM = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP)."""
    src = os.path.join(_HERE, "ocr_oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "ocr_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        # -ffp-contract=off: every operation rounds as written (no fused
        # multiply-add the source does not spell out), in FP64 and FP32 alike
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
                               "-ffp-contract=off", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Forest_(C.Structure):
    _fields_ = [("nleaves", C.c_int), ("max_level", C.c_int),
                ("anchor", C.POINTER(C.c_int32)), ("level", C.POINTER(C.c_uint8)),
                ("nodal", C.POINTER(C.c_float)), ("tf", C.POINTER(C.c_float)),
                ("s_min", C.c_double), ("s_max", C.c_double), ("geometry", C.c_int),
                ("tree", C.POINTER(C.c_int32)), ("frames", C.c_double * 9 * 6),
                ("r0", C.c_double), ("r1", C.c_double)]


class Camera_(C.Structure):
    _fields_ = [("o", C.c_double * 3), ("v", C.c_double * 3), ("t", C.c_double * 3),
                ("u", C.c_double * 3), ("ell", C.c_double), ("near_", C.c_double),
                ("far_", C.c_double), ("w", C.c_int), ("h", C.c_int), ("ortho", C.c_int)]


class Cam32_(C.Structure):
    _fields_ = [("o", C.c_float * 3), ("v", C.c_float * 3), ("lt", C.c_float * 3),
                ("lu", C.c_float * 3), ("t", C.c_float * 3), ("u", C.c_float * 3),
                ("vn", C.c_float * 3), ("n", C.c_float), ("f", C.c_float), ("ell", C.c_float),
                ("cw", C.c_float), ("ch", C.c_float), ("amin", C.c_float), ("amax", C.c_float),
                ("w", C.c_int), ("h", C.c_int), ("ortho", C.c_int)]


class Integrator_(C.Structure):
    _fields_ = [("method", C.c_int), ("nsteps", C.c_int), ("tol", C.c_double),
                ("c_rk", C.c_double), ("max_depth", C.c_int), ("bg", C.c_double * 3),
                ("surface", C.c_int), ("s_iso", C.c_double), ("a_s", C.c_double),
                ("i_s", C.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d = P(C.c_double)
        _lib.orc_combine.argtypes = [d, d, d]
        _lib.orc_inverse.argtypes = [d, d]
        _lib.orc_cut.argtypes = [d, C.c_double, d]
        _lib.orc_average.argtypes = [d, d, d]
        _lib.orc_tf_eval.argtypes = [P(Forest_), C.c_double, d]
        _lib.orc_trilinear.argtypes = [P(C.c_float), C.c_double, C.c_double, C.c_double]
        _lib.orc_trilinear.restype = C.c_double
        _lib.orc_pixel_ray.argtypes = [P(Camera_), C.c_int, C.c_int, d, d, d, d]
        _lib.orc_leaf_rect.argtypes = [P(Forest_), P(Camera_), C.c_int, P(C.c_int32), d,
                                       C.c_double, P(C.c_int)]
        _lib.orc_leaf_rect.restype = C.c_int
        _lib.orc_ray_leaf.argtypes = [P(Forest_), C.c_int, d, d, C.c_double, C.c_double, d, d]
        _lib.orc_ray_leaf.restype = C.c_int
        _lib.orc_ray_leaf_tie.argtypes = [P(Forest_), C.c_int, d, d, C.c_double, C.c_double, d,
                                          d, C.c_double, P(C.c_int)]
        _lib.orc_ray_leaf_tie.restype = C.c_int
        _lib.orc_triquadratic.argtypes = [P(C.c_float), C.c_double, C.c_double, C.c_double]
        _lib.orc_triquadratic.restype = C.c_double
        _lib.orc_shell_map.argtypes = [P(Forest_), C.c_int, d, d]
        _lib.orc_shell_inverse.argtypes = [P(Forest_), C.c_int, d, d]
        _lib.orc_segment_ab.argtypes = [P(Forest_), P(Integrator_), C.c_int, d, d, C.c_double,
                                        C.c_double, d, P(C.c_int64)]
        _lib.orc_cull.argtypes = [P(Forest_), P(Camera_), P(C.c_int32), P(C.c_uint8),
                                  P(C.c_uint8), C.c_double, C.c_int]
        f = P(C.c_float)
        _lib.orc_camera32.argtypes = [P(Camera_), P(Cam32_)]
        _lib.orc_pixel_ray32.argtypes = [P(Cam32_), C.c_int, C.c_int, f, f]
        _lib.orc_shell_tables32.argtypes = [P(Forest_), f, f]
        _lib.orc_leaf_rect32.argtypes = [P(Forest_), P(Cam32_), f, f, C.c_int, P(C.c_int32)]
        _lib.orc_leaf_rect32.restype = C.c_int
        _lib.orc_ray_leaf32.argtypes = [P(Forest_), f, f, C.c_int, f, f, C.c_float, C.c_float,
                                        f, f]
        _lib.orc_ray_leaf32.restype = C.c_int
        _lib.orc_render.argtypes = [P(Forest_), P(Camera_), P(Integrator_), P(C.c_int), C.c_int,
                                    d, P(C.c_int32), P(C.c_uint8), C.c_double, C.c_double,
                                    C.c_int, P(C.c_int64)]
        _lib.orc_render.restype = C.c_int64
        _lib.orc_render_ex.argtypes = [P(Forest_), P(Camera_), P(Integrator_), P(C.c_int),
                                       C.c_int, d, P(C.c_int32), P(C.c_int32), P(C.c_uint8),
                                       C.c_double, C.c_double, C.c_int, P(C.c_int64), C.c_int]
        _lib.orc_render_ex.restype = C.c_int64
        _lib.orc_field_probe.argtypes = [P(Forest_), C.c_int, d, d, C.c_double, C.c_double, d, d]
        _lib.orc_render_grad.argtypes = [P(Forest_), P(Camera_), P(Integrator_), d, d, d, C.c_int,
                                         C.c_int, P(C.c_uint8), C.c_double, d, d]
        _lib.orc_render_grad.restype = C.c_int
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class OracleForest:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, forest, tf):
        if forest.geometry not in ("cube", "shell"):
            raise ValueError(f"oracle forest: unknown geometry {forest.geometry!r}")
        self.anchor = np.ascontiguousarray(forest.anchor, dtype=np.int32)
        self.level = np.ascontiguousarray(forest.level, dtype=np.uint8)
        self.nodal = np.ascontiguousarray(forest.nodal, dtype=np.float32)
        self.tree = np.ascontiguousarray(forest.tree, dtype=np.int32)
        self.tf = np.ascontiguousarray(tf.knots, dtype=np.float32).reshape(-1)
        self.s = Forest_(forest.nleaves, forest.max_level, _ptr(self.anchor, C.c_int32),
                         _ptr(self.level, C.c_uint8), _ptr(self.nodal, C.c_float),
                         _ptr(self.tf, C.c_float), float(tf.s_min), float(tf.s_max))
        self.s.tree = _ptr(self.tree, C.c_int32)
        if forest.geometry == "shell":
            self.s.geometry = 1
            fr = np.asarray(forest.meta["frames"], dtype=np.float64).reshape(-1)
            for k in range(54):
                self.s.frames[k // 9][k % 9] = fr[k]
            self.s.r0, self.s.r1 = float(forest.meta["r0"]), float(forest.meta["r1"])
        self.stride = 27 if forest.geometry == "shell" else 8


def camera_struct(cam) -> Camera_:
    c = Camera_()
    c.o[:] = cam.o
    c.v[:] = cam.v
    c.t[:] = cam.t
    c.u[:] = cam.u
    c.ell, c.near_, c.far_ = cam.ell, cam.near, cam.far
    c.w, c.h, c.ortho = cam.w, cam.h, int(cam.ortho)
    return c


def integrator_struct(integ: dict, bg=(0.0, 0.0, 0.0)) -> Integrator_:
    s = Integrator_()
    if integ["method"] == "rk4":
        s.method, s.nsteps = RK4, int(integ.get("nsteps", 4))
    elif integ["method"] == "dopri5":
        s.method, s.nsteps = DOPRI5, 0
        s.tol = float(integ.get("tol", 1e-6))
        s.c_rk = float(integ.get("c_rk", 0.5))
        s.max_depth = int(integ.get("max_depth", 16))
    elif integ["method"] in ("gauss2", "simpson", "equilibrium"):
        s.method = {"gauss2": GAUSS2, "simpson": SIMPSON, "equilibrium": EQUILIBRIUM}[integ["method"]]
        s.nsteps, s.tol = 0, 0.0
        s.c_rk = float(integ.get("c_rk", 0.5))
        s.max_depth = int(integ.get("max_depth", 16))
    else:
        raise ValueError(integ["method"])
    s.bg[:] = bg
    surf = integ.get("surface")
    if surf:  # Sec. 2.8 on the isosurface s = s_iso: {"s_iso", "a_s", "i_s"}
        s.surface = 1
        s.s_iso, s.a_s = float(surf["s_iso"]), float(surf["a_s"])
        s.i_s[:] = [float(x) for x in surf["i_s"]]
    return s


# -------------------------------------------------------------- primitives --
def combine(near, far):
    out = np.zeros(4)
    lib().orc_combine(_ptr(np.ascontiguousarray(near, float), C.c_double),
                      _ptr(np.ascontiguousarray(far, float), C.c_double), _ptr(out, C.c_double))
    return out


def inverse(s):
    out = np.zeros(4)
    lib().orc_inverse(_ptr(np.ascontiguousarray(s, float), C.c_double), _ptr(out, C.c_double))
    return out


def cut(s, frac):
    out = np.zeros(4)
    lib().orc_cut(_ptr(np.ascontiguousarray(s, float), C.c_double), float(frac),
                  _ptr(out, C.c_double))
    return out


def average(s1, s2):
    out = np.zeros(4)
    lib().orc_average(_ptr(np.ascontiguousarray(s1, float), C.c_double),
                      _ptr(np.ascontiguousarray(s2, float), C.c_double), _ptr(out, C.c_double))
    return out


def tf_eval(of: OracleForest, s: float):
    out = np.zeros(4)
    lib().orc_tf_eval(C.byref(of.s), float(s), _ptr(out, C.c_double))
    return out


def trilinear(nodal8, u, v, w):
    a = np.ascontiguousarray(nodal8, dtype=np.float32)
    return lib().orc_trilinear(_ptr(a, C.c_float), float(u), float(v), float(w))


def triquadratic(nodal27, u, v, w):
    a = np.ascontiguousarray(nodal27, dtype=np.float32)
    return lib().orc_triquadratic(_ptr(a, C.c_float), float(u), float(v), float(w))


def shell_map(of: OracleForest, tree, ref):
    x = np.zeros(3)
    lib().orc_shell_map(C.byref(of.s), int(tree), _ptr(np.ascontiguousarray(ref, float),
                                                       C.c_double), _ptr(x, C.c_double))
    return x


def shell_inverse(of: OracleForest, tree, x):
    ref = np.zeros(3)
    lib().orc_shell_inverse(C.byref(of.s), int(tree), _ptr(np.ascontiguousarray(x, float),
                                                           C.c_double), _ptr(ref, C.c_double))
    return ref


def pixel_ray(cam, i, j):
    org, d, lims = np.zeros(3), np.zeros(3), np.zeros(2)
    cs = camera_struct(cam)
    lib().orc_pixel_ray(C.byref(cs), i, j, _ptr(org, C.c_double), _ptr(d, C.c_double),
                        _ptr(lims[0:1], C.c_double), _ptr(lims[1:2], C.c_double))
    return org, d, float(lims[0]), float(lims[1])


def ray_leaf(of: OracleForest, leaf, org, d, amin, amax):
    """Cube leaf: (hit, alpha_in, alpha_out) of the slab interval."""
    a, b = np.zeros(2), np.zeros(2)
    hit = lib().orc_ray_leaf(C.byref(of.s), int(leaf), _ptr(np.asarray(org, float), C.c_double),
                             _ptr(np.asarray(d, float), C.c_double), float(amin), float(amax),
                             _ptr(a, C.c_double), _ptr(b, C.c_double))
    return bool(hit), float(a[0]), float(b[0])


def ray_leaf_intervals(of: OracleForest, leaf, org, d, amin, amax, band_rel: float = 0.0):
    """All intervals of the ray inside the leaf (at most two), nearest first,
    and the tie flag."""
    a, b = np.zeros(2), np.zeros(2)
    tie = C.c_int(0)
    n = lib().orc_ray_leaf_tie(C.byref(of.s), int(leaf), _ptr(np.asarray(org, float), C.c_double),
                               _ptr(np.asarray(d, float), C.c_double), float(amin), float(amax),
                               _ptr(a, C.c_double), _ptr(b, C.c_double), float(band_rel),
                               C.byref(tie))
    return [(float(a[k]), float(b[k])) for k in range(n)], bool(tie.value)


def field_probe(of: OracleForest, leaf, org, d, a_out, x):
    """Field value and its spatial gradient at alpha = a_out - x / |d| in the leaf."""
    s, g = C.c_double(0.0), np.zeros(3)
    lib().orc_field_probe(C.byref(of.s), int(leaf), _ptr(np.ascontiguousarray(org, float), C.c_double),
                          _ptr(np.ascontiguousarray(d, float), C.c_double), float(a_out), float(x),
                          C.byref(s), _ptr(g, C.c_double))
    return float(s.value), g


def segment_ab(of: OracleForest, integ: dict, leaf, org, d, a_in, a_out):
    out = np.zeros(4)
    st = C.c_int64(0)
    ist = integrator_struct(integ)
    lib().orc_segment_ab(C.byref(of.s), C.byref(ist), int(leaf),
                         _ptr(np.ascontiguousarray(org, float), C.c_double),
                         _ptr(np.ascontiguousarray(d, float), C.c_double), float(a_in),
                         float(a_out), _ptr(out, C.c_double), C.byref(st))
    return out, int(st.value)


def leaf_rect(of: OracleForest, cam, leaf, band_px: float = 0.0):
    """(visible, rect {i0,i1,j0,j1}, projected extents {i_min,i_max,j_min,j_max},
    tie flag) of one leaf."""
    cs = camera_struct(cam)
    rect = np.zeros(4, dtype=np.int32)
    pext = np.zeros(4)
    unc = C.c_int(0)
    vis = lib().orc_leaf_rect(C.byref(of.s), C.byref(cs), int(leaf), _ptr(rect, C.c_int32),
                              _ptr(pext, C.c_double), float(band_px), C.byref(unc))
    return bool(vis), rect, pext, bool(unc.value)


def camera32(cam):
    """The FP32 camera constants of the index decisions (orc_camera32)."""
    k = Cam32_()
    lib().orc_camera32(C.byref(camera_struct(cam)), C.byref(k))
    return k


def shell_tables32(of: OracleForest):
    """FP32 plane tangents and radii of a shell forest (2^L + 1 each)."""
    n = (1 << of.s.max_level) + 1
    tt, rt = np.zeros(n, np.float32), np.zeros(n, np.float32)
    lib().orc_shell_tables32(C.byref(of.s), _ptr(tt, C.c_float), _ptr(rt, C.c_float))
    return tt, rt


def pixel_ray32(k32, i, j):
    org, d = np.zeros(3, np.float32), np.zeros(3, np.float32)
    lib().orc_pixel_ray32(C.byref(k32), int(i), int(j), _ptr(org, C.c_float), _ptr(d, C.c_float))
    return org, d


def leaf_rect32(of: OracleForest, k32, leaf, tables=None):
    """(visible, rect) of one leaf by the FP32 decision."""
    rect = np.zeros(4, dtype=np.int32)
    tt, rt = tables if tables is not None else (None, None)
    vis = lib().orc_leaf_rect32(C.byref(of.s), C.byref(k32),
                                None if tt is None else _ptr(tt, C.c_float),
                                None if rt is None else _ptr(rt, C.c_float), int(leaf),
                                _ptr(rect, C.c_int32))
    return bool(vis), rect


def ray_leaf32(of: OracleForest, leaf, org32, d32, amin, amax, tables=None):
    """FP32 intervals [(a_in, a_out), ...] of the ray in the leaf."""
    a, b = np.zeros(2, np.float32), np.zeros(2, np.float32)
    tt, rt = tables if tables is not None else (None, None)
    o = np.ascontiguousarray(org32, np.float32)
    d = np.ascontiguousarray(d32, np.float32)
    n = lib().orc_ray_leaf32(C.byref(of.s), None if tt is None else _ptr(tt, C.c_float),
                             None if rt is None else _ptr(rt, C.c_float), int(leaf),
                             _ptr(o, C.c_float), _ptr(d, C.c_float), float(amin), float(amax),
                             _ptr(a, C.c_float), _ptr(b, C.c_float))
    return [(float(a[k]), float(b[k])) for k in range(n)]


def cull(forest, tf, cam, band_px: float = 4e-3, decide32: bool = True):
    """Visible flag, pixel rectangle {i0,i1,j0,j1} and tie flag of every leaf.
    decide32 (default): the FP32 decision (no ties flagged); else FP64 with the
    leaves inside the band_px tie band flagged."""
    of = OracleForest(forest, tf)
    cs = camera_struct(cam)
    n = forest.nleaves
    rect = np.zeros((n, 4), dtype=np.int32)
    vis = np.zeros(n, dtype=np.uint8)
    unc = np.zeros(n, dtype=np.uint8)
    lib().orc_cull(C.byref(of.s), C.byref(cs), _ptr(rect, C.c_int32), _ptr(vis, C.c_uint8),
                   _ptr(unc, C.c_uint8), float(band_px), int(bool(decide32)))
    return {"rect": rect, "visible": vis.astype(bool), "uncertain": unc.astype(bool)}


def render(forest, tf, cam, integ: dict, rows=None, bg=(0.0, 0.0, 0.0), nthreads: int = 0,
           band_px: float = 4e-3, band_rel: float = 1e-5, decide32: bool = True):
    """Render the listed rows (default: all).  Returns rgba [nrows, w, 4] (FP64),
    per-ray segment counts, per-ray tie flags and tie counts (leaves of the ray
    with a decision inside the tie band), total segments and RK steps.
    decide32 (default): visibility, rays and intervals by the FP32 decisions,
    values in FP64 (only isosurface sample ties are flagged); else everything
    in FP64 with the geometric ties flagged."""
    of = OracleForest(forest, tf)
    cs = camera_struct(cam)
    ist = integrator_struct(integ, bg)
    if rows is None:
        rows_arr = np.arange(cam.h, dtype=np.int32)
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int32)
    nr = int(rows_arr.shape[0])
    rgba = np.zeros((nr, cam.w, 4), dtype=np.float64)
    counts = np.zeros((nr, cam.w), dtype=np.int32)
    cross = np.zeros((nr, cam.w), dtype=np.int32)
    unc = np.zeros((nr, cam.w), dtype=np.uint8)
    steps = C.c_int64(0)
    total = lib().orc_render_ex(C.byref(of.s), C.byref(cs), C.byref(ist), _ptr(rows_arr, C.c_int),
                                nr, _ptr(rgba, C.c_double), _ptr(counts, C.c_int32),
                                _ptr(cross, C.c_int32), _ptr(unc, C.c_uint8), float(band_px),
                                float(band_rel), int(nthreads), C.byref(steps),
                                int(bool(decide32)))
    if total < 0:
        raise MemoryError("oracle render: allocation failed")
    return {"rgba": rgba, "counts": counts, "crossings": cross, "uncertain": unc.astype(bool),
            "ties": unc.astype(int),
            "segments": int(total), "steps": int(steps.value), "rows": rows_arr}


def render_grad(forest, tf, cam, integ: dict, dL_drgba, bg=(0.0, 0.0, 0.0), nthreads: int = 0,
                decide32: bool = True, tree_band: float | None = None, magnitudes: bool = False):
    """FP64 gradient of L with respect to nodal values [N, 8] (cube) or
    [N, 27] (shell) and knots [8, 4], given dL/d(rgba) [h, w, 4].  With
    tree_band, also the per-leaf flags of DOPRI5 split tests within that
    relative band of their thresholds (another precision may take another
    step tree there).  With magnitudes, also per coordinate the sum of the
    magnitudes of the terms summed into it (nodal, knots): the scale of the
    sum's rounding error in another precision."""
    of = OracleForest(forest, tf)
    cs = camera_struct(cam)
    ist = integrator_struct(integ, bg)
    gb = np.ascontiguousarray(dL_drgba, dtype=np.float64).reshape(cam.h, cam.w, 4)
    gn = np.zeros((forest.nleaves, of.stride))
    gt = np.zeros((8, 4))
    tie = np.zeros(forest.nleaves, np.uint8) if tree_band is not None else None
    an = np.zeros_like(gn) if magnitudes else None
    at = np.zeros_like(gt) if magnitudes else None
    rc = lib().orc_render_grad(C.byref(of.s), C.byref(cs), C.byref(ist), _ptr(gb, C.c_double),
                               _ptr(gn, C.c_double), _ptr(gt, C.c_double), int(nthreads),
                               int(bool(decide32)), None if tie is None else _ptr(tie, C.c_uint8),
                               float(tree_band or 0.0),
                               None if an is None else _ptr(an, C.c_double),
                               None if at is None else _ptr(at, C.c_double))
    if rc == -1:
        raise MemoryError("oracle gradient: allocation failed")
    if rc != 0:
        raise ValueError("oracle gradient: surfaces are not differentiated")
    out = (gn, gt)
    if tree_band is not None:
        out += (tie.astype(bool),)
    if magnitudes:
        out += (an, at)
    return out
