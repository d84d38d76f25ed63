"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Images: max |delta| <= 1e-4 per RGBA channel.  Index results (visible-leaf
set, pixel rectangles, per-ray segment counts): bit-exact on every leaf and
every ray.  Both sides take those decisions in FP32, the kernels' precision,
by the same canonical evaluation (the oracle's orc_*32 functions, pinned to
the FP64 definitions in tests/test_oracle_fp32_decisions.py); the segment
values are the oracle's FP64 integration.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _renderer(forest, tf, integ, cam, bg=(0.0, 0.0, 0.0)):
    from paper_1809_01334_gb300 import Renderer
    r = Renderer(forest, tf, integ, bg=bg)
    r.set_camera(cam)
    return r


def _compare(forest, tf, cam, integ, rows=None, bg=(0.0, 0.0, 0.0)):
    r = _renderer(forest, tf, integ, cam, bg)
    img, st = r.render(with_index=True)
    torch.cuda.synchronize()
    ref = O.render(forest, tf, cam, integ, rows=rows, bg=bg)
    rr = ref["rows"]
    got = img.cpu().numpy().astype(np.float64)[rr]
    dev = np.abs(got - ref["rgba"])
    err = dev.max()
    if err > TOL:
        j, i, c = np.unravel_index(np.argmax(dev), dev.shape)
        raise AssertionError(f"max |delta| = {err:.3e} at row {rr[j]} column {i} channel {c}: "
                             f"GPU {got[j, i]} oracle {ref['rgba'][j, i]}, segments "
                             f"{int(st['counts'][rr[j], i])} / {int(ref['counts'][j, i])}")
    counts = st["counts"].cpu().numpy()[rr]
    bad = counts != ref["counts"]
    assert not bad.any(), f"{int(bad.sum())} of {bad.size} rays with different segment counts"
    cull = O.cull(forest, tf, cam)
    vis = st["visible"].cpu().numpy().astype(bool)
    np.testing.assert_array_equal(vis, cull["visible"])
    np.testing.assert_array_equal(st["rects"].cpu().numpy(), cull["rect"])
    if rows is None:
        assert st["segments"] == int(counts.sum())
        assert st["visible_leaves"] == int(vis.sum())
    r.close()
    return err, st, ref


def test_c1_uniform_orthographic_rk4():
    """C1: 512 leaves, orthographic 64x64, RK4 x 4: every ray has 8 segments."""
    f, tf, cam, integ = I.preset_c1()
    err, st, ref = _compare(f, tf, cam, integ)
    assert st["segments"] == 64 * 64 * 8 and st["visible_leaves"] == 512
    assert st["rk_steps"] == 64 * 64 * 8 * 4


@pytest.mark.parametrize("integ", [{"method": "rk4", "nsteps": 4},
                                   {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}])
def test_small_adaptive_perspective(integ):
    """Adaptive 2:1-balanced mesh (levels 3-4), perspective 48x40 image."""
    f, tf, cam = I.preset_small()
    _compare(f, tf, cam, integ)


@pytest.mark.parametrize("integ", [{"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
                                   {"method": "simpson", "c_rk": 0.2, "max_depth": 16},
                                   {"method": "equilibrium", "c_rk": 0.2, "max_depth": 16}])
def test_gauss2_and_simpson_integrators(integ):
    """Sec. 2.7's implicit Gauss closed form and Simpson quadrature, and the
    intensity interface of Eq. 2.18, inside Algorithm 1, on the adaptive mesh
    with a non-zero background."""
    f, tf, cam = I.preset_small(w=64, h=48)
    _compare(f, tf, cam, integ, bg=(0.1, 0.2, 0.3))


@pytest.mark.parametrize("shape", [(37, 23), (1, 1), (129, 3), (5, 97)])
def test_ragged_images(shape):
    """Image sizes that are not multiples of any tile, including 1x1.  With an
    odd width the centre column of this target-centred camera (up = +z) runs
    exactly through the grid edge x = y = 1/2, and the 1x1 ray through the
    cube's centre vertex: exact geometric ties, which the FP32 decisions of
    both sides still take identically."""
    f, tf, cam = I.preset_small(w=shape[0], h=shape[1], cam_seed=3)
    _compare(f, tf, cam, {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16})


def test_adaptive_levels_1_to_5_with_background():
    fld = I.gaussian_field(16, 99)
    f = I.adaptive_cube_forest(fld, 1, 5, 0.3, balance=True)
    assert len(np.unique(f.level)) >= 3
    tf = I.transfer_function(f.nodal, 5)
    cam = I.perspective_camera(21, 64, 48, dist=(1.6, 2.0))
    _compare(f, tf, cam, {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16},
             bg=(0.3, 0.2, 0.1))


def test_single_leaf_forest_and_empty_view():
    fld = I.gaussian_field(4, 1809)
    f = I.uniform_cube_forest(0, fld)
    tf = I.transfer_function(f.nodal)
    cam = I.perspective_camera(7, 20, 16, dist=(1.5, 1.6))
    _compare(f, tf, cam, {"method": "rk4", "nsteps": 8})
    # a camera looking away from the cube: background everywhere, nothing visible
    away = I.Camera(o=(0.5, 0.5, 3.0), v=(0.0, 0.0, 0.1), t=(1.0, 0, 0), u=(0, 1.0, 0),
                    ell=0.001, near=0.1, far=100.0, w=16, h=8)
    f2, tf2, _ = I.preset_small()
    r = _renderer(f2, tf2, {"method": "rk4", "nsteps": 4}, away, bg=(0.5, 0.25, 0.125))
    img, st = r.render(with_index=True)
    assert st["segments"] == 0 and st["visible_leaves"] == 0
    np.testing.assert_array_equal(img.cpu().numpy().reshape(-1, 4),
                                  np.tile([0.5, 0.25, 0.125, 0.0], (16 * 8, 1)))


def test_deterministic():
    f, tf, cam = I.preset_small()
    r = _renderer(f, tf, {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}, cam)
    a, _ = r.render()
    a = a.clone()
    b, _ = r.render()
    assert torch.equal(a, b)


def test_c2_full_size_whole_image():
    """C2 at its full size (2,053,451 leaves, 1920x1080, DOPRI5 tol 1e-6) in
    the launch configuration the benchmark times: every pixel of the image
    against the oracle, and the segment total against the sum of the
    oracle's per-ray counts."""
    f, tf, cam, integ = I.preset_c2()
    err, st, ref = _compare(f, tf, cam, integ)
    assert st["visible_leaves"] == f.nleaves
    assert st["segments"] > 20_000_000


def _spike_forest(max_level, p=(0.3137, 0.5821, 0.4419), seed=5):
    """A forest refined only around the point p, one cell per level, down to
    max_level: 7 leaves per level and 8 at the finest (Morton order)."""
    L = max_level
    levels, anchors = [], []
    cell = np.zeros(3, np.int64)  # anchor (units of 2^-L) of the refined cell at each level
    for l in range(L):
        half = 1 << (L - l - 1)
        pc = np.floor(np.asarray(p) * (1 << (l + 1))).astype(np.int64) & 1  # child holding p
        for o in range(8):
            bits = np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1])
            a = cell + bits * half
            if l + 1 < L and (bits == pc).all():
                continue
            levels.append(l + 1)
            anchors.append(a)
        cell = cell + pc * half
    lv = np.array(levels, np.uint8)
    an = np.array(anchors, np.int32)
    lv, an, tr = I._sort_forest(lv, an, np.zeros(len(lv), np.int32))
    fld = I.gaussian_field(4, seed)
    nodal = I._sample_corners(fld, lv, an, L).astype(np.float32)
    f = I.Forest("cube", L, lv, an, tr, nodal, {"kind": "spike"})
    tf = I.transfer_function(f.nodal, 1334)
    return f, tf


@pytest.mark.parametrize("max_level", [12, 16])
def test_deep_forest_zoomed_camera(max_level):
    """Maximum depths: a forest refined around one point to level 12 and 16
    (anchors up to 2^16), seen by a camera zoomed onto that point so that the
    deep cells cover pixels; 13 coarsening passes above the tile level."""
    f, tf = _spike_forest(max_level)
    assert f.nleaves == 7 * max_level + 1
    p = (0.3137, 0.5821, 0.4419)
    cam = I.perspective_camera(13, 40, 32, dist=(2e-3, 2.5e-3), fov_deg=30.0, near=1e-4,
                               target=p)
    err, st, ref = _compare(f, tf, cam, {"method": "rk4", "nsteps": 4})
    assert (ref["counts"] > 0).all() and st["visible_leaves"] >= max_level


def test_wide_image_index_arithmetic():
    """A 4096 x 7 image: pixel and slot indices across a wide row."""
    f, tf, _ = I.preset_small()
    cam = I.perspective_camera(17, 4096, 7)
    _compare(f, tf, cam, {"method": "rk4", "nsteps": 2})


def test_render_host_equals_device_render():
    """ocr_render_host (host data in, host image out, the copy overlapping the
    pruning) gives the device render's pixels bit for bit, for a cube and a
    shell forest, and leaves the library's copy as the renderer's data."""
    from paper_1809_01334_gb300 import Renderer
    integ = {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16}
    for f, tf, cam in (I.preset_small("adaptive"), I.preset_shell_small()):
        r = Renderer(f, tf, integ)
        r.set_camera(cam)
        ref, _ = r.render()
        ref = ref.cpu()
        nodal_h = torch.from_numpy(np.ascontiguousarray(f.nodal, np.float32)).pin_memory()
        tf_h = torch.from_numpy(np.ascontiguousarray(tf.knots, np.float32)).pin_memory()
        out_h = torch.empty((cam.h, cam.w, 4), dtype=torch.float32).pin_memory()
        st = r.render_host(nodal_h, tf_h, out_h)
        assert st["launches"] > 0
        assert torch.equal(out_h, ref)
        again, _ = r.render()  # now from the library's device copy
        assert torch.equal(again.cpu(), ref)
        r.close()
