"""CPU checks of the CUDA library's C ABI: it builds, loads, exports every
entry point include/ocraycast.h declares, and rejects malformed forests and
arguments on the host before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1809_01334_gb300 import build as B
from paper_1809_01334_gb300 import capi
from paper_1809_01334_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.lib()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ocr_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert "ocr_render" in names and "ocr_build_forest" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(capi.EXPORTS) <= set(names)


def test_strerror(lib):
    assert capi.strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6):
        assert capi.strerror(code) not in ("ok", "unknown error")
    assert capi.strerror(-99) == "unknown error"


def _desc(level, anchor, L, geometry=0):
    lv = np.ascontiguousarray(level, np.uint8)
    an = np.ascontiguousarray(anchor, np.int32)
    d = capi.ForestDesc(geometry, L, lv.shape[0], an.ctypes.data_as(C.POINTER(C.c_int32)),
                        lv.ctypes.data_as(C.POINTER(C.c_uint8)))
    return d, (lv, an)


def _build_rc(lib, level, anchor, L, geometry=0):
    d, keep = _desc(level, anchor, L, geometry)
    h = C.c_void_p()
    rc = lib.ocr_build_forest(C.byref(d), None, C.byref(h))
    if rc == 0:
        lib.ocr_destroy(h)
    return rc


def test_malformed_forests_are_rejected_on_the_host(lib):
    f = I.uniform_cube_forest(2, I.gaussian_field(4, 1))
    lv, an = f.level, f.anchor
    # out of Morton order
    perm = np.arange(f.nleaves)
    perm[[3, 4]] = perm[[4, 3]]
    assert _build_rc(lib, lv[perm], an[perm], f.max_level) == capi.ERR_INVALID
    # a gap (leaf removed)
    assert _build_rc(lib, lv[1:], an[1:], f.max_level) == capi.ERR_INVALID
    # an overlap (leaf duplicated)
    assert _build_rc(lib, np.r_[lv[:1], lv], np.r_[an[:1], an], f.max_level) == capi.ERR_INVALID
    # level above max_level, misaligned anchor, negative anchor
    bad = lv.copy(); bad[0] = 3
    assert _build_rc(lib, bad, an, 2) == capi.ERR_INVALID
    an2 = an.copy(); an2[5, 0] += 1
    assert _build_rc(lib, lv, an2, f.max_level) == capi.ERR_INVALID
    an3 = an.copy(); an3[0, 2] = -4
    assert _build_rc(lib, lv, an3, f.max_level) == capi.ERR_INVALID
    # unsupported geometry, absurd max_level
    assert _build_rc(lib, lv, an, f.max_level, geometry=7) == capi.ERR_UNSUPPORTED
    assert _build_rc(lib, lv, an, 25) == capi.ERR_INVALID


def _shell_rc(lib, f, tree=None, frames=None, r0=None, r1=None, level=None, anchor=None):
    lv = np.ascontiguousarray(f.level if level is None else level, np.uint8)
    an = np.ascontiguousarray(f.anchor if anchor is None else anchor, np.int32)
    tr = np.ascontiguousarray(f.tree if tree is None else tree, np.int32)
    d = capi.ForestDesc(capi.GEOM_SHELL, f.max_level, lv.shape[0],
                        an.ctypes.data_as(C.POINTER(C.c_int32)),
                        lv.ctypes.data_as(C.POINTER(C.c_uint8)))
    d.h_tree = tr.ctypes.data_as(C.POINTER(C.c_int32))
    fr = np.asarray(f.meta["frames"] if frames is None else frames, np.float64).reshape(6, 9)
    for t in range(6):
        for k in range(9):
            d.frames[t][k] = float(fr[t, k])
    d.r0 = f.meta["r0"] if r0 is None else r0
    d.r1 = f.meta["r1"] if r1 is None else r1
    h = C.c_void_p()
    rc = lib.ocr_build_forest(C.byref(d), None, C.byref(h))
    if rc == 0:
        lib.ocr_destroy(h)
    return rc


def test_malformed_shell_forests_are_rejected_on_the_host(lib):
    f = I.shell_forest(I.shell_noise(1809, 8), 1, 2, 2.0)
    fr = np.asarray(f.meta["frames"], np.float64)
    # frames: a tilted normal, two trees around the same axis direction, a repeated axis
    bad = fr.copy(); bad[0, 0] = [0.6, 0.8, 0.0]
    assert _shell_rc(lib, f, frames=bad) == capi.ERR_INVALID
    bad = fr.copy(); bad[1] = bad[0]
    assert _shell_rc(lib, f, frames=bad) == capi.ERR_INVALID
    bad = fr.copy(); bad[2, 1] = bad[2, 0]
    assert _shell_rc(lib, f, frames=bad) == capi.ERR_INVALID
    # radii, tree ids out of range or out of order, a tree left incomplete
    assert _shell_rc(lib, f, r0=0.0) == capi.ERR_INVALID
    assert _shell_rc(lib, f, r0=1.2, r1=1.0) == capi.ERR_INVALID
    tr = f.tree.copy(); tr[0] = 6
    assert _shell_rc(lib, f, tree=tr) == capi.ERR_INVALID
    tr = f.tree.copy(); tr[-1] = 4
    assert _shell_rc(lib, f, tree=tr) == capi.ERR_INVALID
    keep = f.tree != 3
    assert _shell_rc(lib, f, tree=f.tree[keep], level=f.level[keep],
                     anchor=f.anchor[keep]) == capi.ERR_INVALID
    # a gap inside a tree
    drop = np.ones(f.nleaves, bool); drop[np.flatnonzero(f.tree == 2)[3]] = False
    assert _shell_rc(lib, f, tree=f.tree[drop], level=f.level[drop],
                     anchor=f.anchor[drop]) == capi.ERR_INVALID


def test_null_handles_are_rejected(lib):
    integ = capi.Integrator(0, 4, 1e-6, 0.5, 16)
    assert lib.ocr_set_integrator(None, C.byref(integ)) == capi.ERR_INVALID
    cam = capi.Camera()
    assert lib.ocr_set_camera(None, C.byref(cam), 1) == capi.ERR_INVALID
    assert lib.ocr_render(None, None, None, None) == capi.ERR_INVALID
    buf = np.zeros(64, np.float32)
    assert lib.ocr_render_host(None, buf.ctypes.data, buf.ctypes.data, 0.0, 1.0,
                               buf.ctypes.data, None, None) == capi.ERR_INVALID
    assert lib.ocr_render_backward(None, None, None, None, None) == capi.ERR_INVALID
    assert lib.ocr_forest_set_data(None, None, None, 0.0, 1.0, None) == capi.ERR_INVALID
    assert lib.ocr_device_bytes(None) == 0
    t = capi.Tuning(3, 4, 0, 0, 1, 1, 0, 0.0)
    lib.ocr_set_tuning.argtypes = [C.c_void_p, C.POINTER(capi.Tuning)]
    assert lib.ocr_set_tuning(None, C.byref(t)) == capi.ERR_INVALID
    lib.ocr_autotune.argtypes = [C.c_void_p, C.c_int, C.POINTER(capi.Tuning),
                                 C.POINTER(capi.Tuning), C.c_int, C.POINTER(C.c_int)]
    assert lib.ocr_autotune(None, 3, C.byref(t), None, 0, None) == capi.ERR_INVALID
    lib.ocr_destroy(None)
