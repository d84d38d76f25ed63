"""ctypes binding of the C ABI in include/ocraycast.h (argument marshalling only).

Every function here has the name of the C entry point without the ``ocr_``
prefix and does nothing but convert arguments: the whole render path runs in
the CUDA library ``_build/libocraycast.so``.  If that library is missing this
module raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libocraycast.so")

OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_UNSUPPORTED, ERR_DEVICE, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
GEOM_CUBE, GEOM_SHELL = 0, 1
RK4, DOPRI5, GAUSS2, SIMPSON, EQUILIBRIUM = 0, 1, 2, 3, 4

EXPORTS = ["ocr_build_forest", "ocr_forest_set_data", "ocr_set_integrator", "ocr_set_camera",
           "ocr_render", "ocr_render_view", "ocr_render_host", "ocr_render_backward",
           "ocr_set_tuning", "ocr_get_tuning", "ocr_autotune", "ocr_prune_noalloc",
           "ocr_device_bytes", "ocr_destroy", "ocr_strerror", "ocr_sync", "ocr_fold_segments"]


class ForestDesc(C.Structure):
    _fields_ = [("geometry", C.c_int), ("max_level", C.c_int), ("nleaves", C.c_int64),
                ("h_anchor", C.POINTER(C.c_int32)), ("h_level", C.POINTER(C.c_uint8)),
                ("h_tree", C.POINTER(C.c_int32)), ("frames", C.c_double * 9 * 6),
                ("r0", C.c_double), ("r1", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("o", C.c_double * 3), ("v", C.c_double * 3), ("t", C.c_double * 3),
                ("u", C.c_double * 3), ("ell", C.c_double), ("near_", C.c_double),
                ("far_", C.c_double), ("w", C.c_int), ("h", C.c_int), ("ortho", C.c_int)]


class Integrator(C.Structure):
    _fields_ = [("method", C.c_int), ("nsteps", C.c_int), ("tol", C.c_float), ("c_rk", C.c_float),
                ("max_depth", C.c_int), ("bg", C.c_float * 3), ("surface", C.c_int),
                ("s_iso", C.c_float), ("a_s", C.c_float), ("i_s", C.c_float * 3)]


class Stats(C.Structure):
    _fields_ = [("d_counts", C.c_void_p), ("d_visible", C.c_void_p), ("d_rects", C.c_void_p),
                ("fill_counters", C.c_int), ("time_phases", C.c_int),
                ("visible_leaves", C.c_int64), ("segments", C.c_int64), ("rk_steps", C.c_int64),
                ("leaf_tests", C.c_int64), ("slots", C.c_int64),
                ("subtree_segments", C.c_int64), ("subtree_rk_steps", C.c_int64),
                ("subtree_node_visits", C.c_int64),
                ("launches", C.c_int64), ("ms_prune", C.c_float), ("ms_merge", C.c_float),
                ("ms_subtree", C.c_float)]


class Tuning(C.Structure):
    _fields_ = [("tile_depth", C.c_int), ("streams", C.c_int), ("shell_warps", C.c_int),
                ("merge", C.c_int), ("persistent", C.c_int), ("chunks_per_item", C.c_int),
                ("ctas_per_sm", C.c_int), ("ms", C.c_float)]


class OcrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.ocr_build_forest.argtypes = [C.POINTER(ForestDesc), vp, C.POINTER(vp)]
        L.ocr_forest_set_data.argtypes = [vp, vp, vp, C.c_float, C.c_float, vp]
        L.ocr_set_integrator.argtypes = [vp, C.POINTER(Integrator)]
        L.ocr_set_camera.argtypes = [vp, C.POINTER(Camera), C.c_int]
        L.ocr_render.argtypes = [vp, vp, vp, C.POINTER(Stats)]
        L.ocr_render_view.argtypes = [vp, C.c_int, vp, vp, C.POINTER(Stats)]
        L.ocr_render_host.argtypes = [vp, vp, vp, C.c_float, C.c_float, vp, vp,
                                      C.POINTER(Stats)]
        L.ocr_device_bytes.argtypes = [vp]
        L.ocr_device_bytes.restype = C.c_int64
        L.ocr_destroy.argtypes = [vp]
        L.ocr_destroy.restype = None
        L.ocr_strerror.argtypes = [C.c_int]
        L.ocr_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().ocr_strerror(int(code)).decode()
    except Exception:  # the library itself is unavailable
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != OK:
        raise OcrError(rc, what)


def _ptr(x):
    """Device or host address of a tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def build_forest(level, anchor, max_level: int, stream=None, geometry: int = GEOM_CUBE,
                 tree=None, frames=None, r0: float = 0.0, r1: float = 0.0):
    """ocr_build_forest.  level: uint8 [N], anchor: int32 [N, 3] (host numpy);
    shell forests also tree: int32 [N], frames: [6, 3, 3] (rows n, e1, e2), r0, r1."""
    import numpy as np
    lv = np.ascontiguousarray(level, dtype=np.uint8)
    an = np.ascontiguousarray(anchor, dtype=np.int32)
    d = ForestDesc(geometry, int(max_level), int(lv.shape[0]),
                   an.ctypes.data_as(C.POINTER(C.c_int32)), lv.ctypes.data_as(C.POINTER(C.c_uint8)))
    if geometry == GEOM_SHELL:
        tr = np.ascontiguousarray(tree, dtype=np.int32)
        d.h_tree = tr.ctypes.data_as(C.POINTER(C.c_int32))
        fr = np.asarray(frames, dtype=np.float64).reshape(6, 9)
        for t in range(6):
            for k in range(9):
                d.frames[t][k] = float(fr[t, k])
        d.r0, d.r1 = float(r0), float(r1)
    h = C.c_void_p()
    _check(lib().ocr_build_forest(C.byref(d), _ptr(stream), C.byref(h)), "ocr_build_forest")
    return h


def forest_set_data(h, d_nodal, d_tf, s_min: float, s_max: float, stream=None):
    _check(lib().ocr_forest_set_data(h, _ptr(d_nodal), _ptr(d_tf), float(s_min), float(s_max),
                                     _ptr(stream)), "ocr_forest_set_data")


def set_integrator(h, method: int, nsteps: int = 4, tol: float = 1e-6, c_rk: float = 0.5,
                   max_depth: int = 16, bg=(0.0, 0.0, 0.0), surface=None):
    """surface: None, or {"s_iso", "a_s", "i_s"} for the isosurface of Sec. 2.8."""
    s = Integrator(int(method), int(nsteps), float(tol), float(c_rk), int(max_depth))
    s.bg[:] = bg
    if surface:
        s.surface = 1
        s.s_iso, s.a_s = float(surface["s_iso"]), float(surface["a_s"])
        s.i_s[:] = [float(x) for x in surface["i_s"]]
    _check(lib().ocr_set_integrator(h, C.byref(s)), "ocr_set_integrator")


def set_camera(h, o, v, t, u, ell, near, far, w, h_px, ortho=False):
    c = Camera()
    c.o[:], c.v[:], c.t[:], c.u[:] = o, v, t, u
    c.ell, c.near_, c.far_ = float(ell), float(near), float(far)
    c.w, c.h, c.ortho = int(w), int(h_px), int(bool(ortho))
    _check(lib().ocr_set_camera(h, C.byref(c), 1), "ocr_set_camera")


def set_cameras(h, cams):
    """ocr_set_camera with several cameras (inputs.Camera objects)."""
    arr = (Camera * len(cams))()
    for c, cam in zip(arr, cams):
        c.o[:], c.v[:], c.t[:], c.u[:] = cam.o, cam.v, cam.t, cam.u
        c.ell, c.near_, c.far_ = float(cam.ell), float(cam.near), float(cam.far)
        c.w, c.h, c.ortho = int(cam.w), int(cam.h), int(bool(cam.ortho))
    _check(lib().ocr_set_camera(h, arr, len(cams)), "ocr_set_camera")


def render(h, d_rgba, stream=None, d_counts=None, d_visible=None, d_rects=None,
           fill_counters: bool = False, time_phases: bool = False) -> dict:
    s = Stats(_ptr(d_counts), _ptr(d_visible), _ptr(d_rects), int(bool(fill_counters)),
              int(bool(time_phases)))
    _check(lib().ocr_render(h, _ptr(d_rgba), _ptr(stream), C.byref(s)), "ocr_render")
    return {"visible_leaves": s.visible_leaves, "segments": s.segments, "rk_steps": s.rk_steps,
            "leaf_tests": s.leaf_tests, "slots": s.slots,
            "subtree_segments": s.subtree_segments, "subtree_rk_steps": s.subtree_rk_steps,
            "subtree_node_visits": s.subtree_node_visits,
            "launches": s.launches, "ms_prune": s.ms_prune, "ms_merge": s.ms_merge,
            "ms_subtree": s.ms_subtree}


def render_view(h, view: int, d_rgba, stream=None, d_counts=None, fill_counters: bool = False,
                time_phases: bool = False) -> dict:
    """ocr_render_view: one camera of the last set_cameras, alone, into its own image."""
    s = Stats(_ptr(d_counts), None, None, int(bool(fill_counters)), int(bool(time_phases)))
    _check(lib().ocr_render_view(h, int(view), _ptr(d_rgba), _ptr(stream), C.byref(s)),
           "ocr_render_view")
    return {"segments": s.segments, "rk_steps": s.rk_steps, "launches": s.launches,
            "ms_prune": s.ms_prune, "ms_merge": s.ms_merge, "ms_subtree": s.ms_subtree}


def render_host(h, h_nodal, h_tf, s_min: float, s_max: float, h_rgba, stream=None) -> dict:
    """ocr_render_host: host field and knots in, host image out (blocks)."""
    for a in (h_nodal, h_tf, h_rgba):
        if hasattr(a, "device") and a.device.type != "cpu":
            raise ValueError("ocr_render_host takes host buffers")
    s = Stats()
    _check(lib().ocr_render_host(h, _ptr(h_nodal), _ptr(h_tf), float(s_min), float(s_max),
                                 _ptr(h_rgba), _ptr(stream), C.byref(s)), "ocr_render_host")
    return {"segments": s.segments, "rk_steps": s.rk_steps, "launches": s.launches}


def _tuning_dict(t: Tuning) -> dict:
    return {"tile_depth": t.tile_depth, "streams": t.streams, "shell_warps": t.shell_warps,
            "merge": t.merge, "persistent": t.persistent, "chunks_per_item": t.chunks_per_item,
            "ctas_per_sm": t.ctas_per_sm, "ms": float(t.ms)}


def set_tuning(h, tile_depth: int = 4, streams: int = 4, shell_warps: int = 0, merge: int = 1,
               persistent: int = 1, chunks_per_item: int = 16, ctas_per_sm: int = 0):
    """ocr_set_tuning (a cube forest re-plans its cameras when tile_depth changes)."""
    t = Tuning(int(tile_depth), int(streams), int(shell_warps), int(merge), int(persistent),
               int(chunks_per_item), int(ctas_per_sm), 0.0)
    L = lib()
    L.ocr_set_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
    _check(L.ocr_set_tuning(h, C.byref(t)), "ocr_set_tuning")


def get_tuning(h) -> dict:
    t = Tuning()
    L = lib()
    L.ocr_get_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
    _check(L.ocr_get_tuning(h, C.byref(t)), "ocr_get_tuning")
    return _tuning_dict(t)


def autotune(h, reps: int = 3) -> dict:
    """ocr_autotune: times every candidate tuning on the current cameras and
    keeps the fastest.  Returns {"best": ..., "tried": [...]}."""
    best = Tuning()
    tried = (Tuning * 128)()
    n = C.c_int(0)
    L = lib()
    L.ocr_autotune.argtypes = [C.c_void_p, C.c_int, C.POINTER(Tuning), C.POINTER(Tuning), C.c_int,
                               C.POINTER(C.c_int)]
    _check(L.ocr_autotune(h, int(reps), C.byref(best), tried, 128, C.byref(n)), "ocr_autotune")
    return {"best": _tuning_dict(best), "tried": [_tuning_dict(tried[k]) for k in range(n.value)]}


def device_bytes(h) -> int:
    return int(lib().ocr_device_bytes(h))


def destroy(h):
    if h:
        lib().ocr_destroy(h)


def prune_noalloc(d_leaf_geo, nleaves: int, max_level: int, cam, d_rects, d_visible_idx,
                  stream=None) -> int:
    """ocr_prune_noalloc: pruning without any device allocation (for callers
    that cannot allocate when they need the result).  Returns the number of
    visible leaves; d_visible_idx[:n] holds their indices in Morton order."""
    L = lib()
    fn = L.ocr_prune_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.POINTER(Camera), C.c_void_p, C.c_void_p,
                   C.POINTER(C.c_int64), C.c_void_p]
    c = Camera()
    c.o[:], c.v[:], c.t[:], c.u[:] = cam.o, cam.v, cam.t, cam.u
    c.ell, c.near_, c.far_ = float(cam.ell), float(cam.near), float(cam.far)
    c.w, c.h, c.ortho = int(cam.w), int(cam.h), int(bool(cam.ortho))
    n = C.c_int64(-1)
    _check(fn(_ptr(d_leaf_geo), int(nleaves), int(max_level), C.byref(c), _ptr(d_rects),
              _ptr(d_visible_idx), C.byref(n), _ptr(stream)), "ocr_prune_noalloc")
    return int(n.value)


def render_backward(h, d_dL_drgba, d_grad_nodal, d_grad_tf, stream=None):
    """ocr_render_backward: dL/d(nodal) and dL/d(knots) given dL/d(rgba)."""
    fn = lib().ocr_render_backward
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    _check(fn(h, _ptr(d_dL_drgba), _ptr(d_grad_nodal), _ptr(d_grad_tf), _ptr(stream)),
           "ocr_render_backward")


def fold_segments(d_val, d_iv, d_out, stream=None):
    """ocr_fold_segments: the shell's per-ray merge (Eq. 2.14; cut and average of
    overlaps, Eqs. 2.20-2.21) of one list: d_val [n, 4], d_iv [n, 2] -> d_out [4]."""
    fn = lib().ocr_fold_segments
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    _check(fn(_ptr(d_val), _ptr(d_iv), int(d_val.shape[0]), _ptr(d_out), _ptr(stream)),
           "ocr_fold_segments")


def sync(h, stream=None):
    """ocr_sync: wait for the stream; raise if a stream-ordered call recorded a device error."""
    fn = lib().ocr_sync
    fn.argtypes = [C.c_void_p, C.c_void_p]
    _check(fn(h, _ptr(stream)), "ocr_sync")
