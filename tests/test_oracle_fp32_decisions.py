"""Pins of the oracle's FP32 index decisions.

Visibility, pixel rectangles and per-ray segments are decided by floating
point; the oracle takes those decisions in FP32, the GPU path's precision,
with one canonical evaluation (orc_camera32, orc_pixel_ray32, orc_leaf_rect32,
orc_ray_leaf32).  These tests tie that FP32 code to the FP64 definitions it
evaluates (which the closed-form and brute-force pins in test_oracle_pins.py
and test_oracle_shell_pins.py hold to the paper): the same decisions wherever
the FP64 decision is not within its tie band, end points within a few FP32
rounding errors, conservative rectangles, and images that agree to FP32
accuracy.  A slip in the FP32 code (a swapped plane, a wrong sign, a dropped
term) breaks the agreement on many pairs at once.
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_01334_gb300 import inputs as I

EPS32 = 2.0 ** -24


def _cases():
    fld = I.gaussian_field(16, 99)
    f = I.adaptive_cube_forest(fld, 1, 3, 0.3, balance=True)
    yield "cube", f, I.transfer_function(f.nodal), I.perspective_camera(21, 12, 9, dist=(1.6, 2.0))
    f, tf, _ = I.preset_shell_small(max_level=2)
    yield "shell", f, tf, I.perspective_camera(4, 12, 9, dist=(2.0, 2.4), target=(0.0, 0.0, 0.0))
    f = I.uniform_cube_forest(2, I.gaussian_field(4, 1809))
    yield "ortho", f, I.transfer_function(f.nodal), I.ortho_camera_c1(8, 8)  # centres off faces


@pytest.fixture(scope="module", params=["cube", "shell", "ortho"])
def case(request):
    for name, f, tf, cam in _cases():
        if name == request.param:
            return name, f, tf, cam
    raise KeyError(request.param)


def test_fp32_camera_is_the_fp64_camera_rounded_once(case):
    """Step a1: every FP32 ray constant is its FP64 value rounded once."""
    _, f, tf, cam = case
    k = O.camera32(cam)
    n = cam.near
    v = np.asarray(cam.v) / n if cam.ortho else np.asarray(cam.v)
    for got, want in ((k.o, cam.o), (k.v, v), (k.lt, cam.ell * np.asarray(cam.t)),
                      (k.lu, cam.ell * np.asarray(cam.u)), (k.vn, np.asarray(cam.v) / n)):
        np.testing.assert_array_equal(np.array(got[:], np.float32), np.float32(want))
    assert k.amax == np.float32(cam.far if cam.ortho else cam.far / n)
    assert (k.cw, k.ch) == ((cam.w - 1) / 2, (cam.h - 1) / 2)


def test_fp32_rays_are_the_fp64_rays_to_rounding(case):
    _, f, tf, cam = case
    k = O.camera32(cam)
    for j in range(cam.h):
        for i in range(cam.w):
            o64, d64, amin, amax = O.pixel_ray(cam, i, j)
            o32, d32 = O.pixel_ray32(k, i, j)
            assert np.abs(o32 - o64).max() <= 4 * EPS32 * (np.abs(o64).max() + 1.0)
            assert np.abs(d32 - d64).max() <= 4 * EPS32 * np.abs(d64).max()


def test_fp32_rectangles_match_fp64_outside_the_tie_band(case):
    _, f, tf, cam = case
    c64 = O.cull(f, tf, cam, band_px=1e-3, decide32=False)
    c32 = O.cull(f, tf, cam)
    assert not c32["uncertain"].any()
    same = (c64["rect"] == c32["rect"]).all(axis=1)
    assert not (~same & ~c64["uncertain"]).any()
    assert not ((c64["visible"] != c32["visible"]) & ~c64["uncertain"]).any()
    assert c32["visible"].sum() > 0


def test_fp32_intervals_match_fp64_outside_the_tie_band(case):
    """Every (leaf, ray) pair of the image: the FP32 intervals have the FP64
    decision's number of pieces unless the FP64 decision is within 1e-6 of
    flipping, and their end points are within 32 FP32 rounding errors (the
    crossings are short chains of rounded operations); an FP32 hit always lies
    inside the leaf's FP32 rectangle (the GPU tests only those pairs)."""
    name, f, tf, cam = case
    of = O.OracleForest(f, tf)
    k = O.camera32(cam)
    tabs = O.shell_tables32(of) if f.geometry == "shell" else None
    rect = O.cull(f, tf, cam)["rect"]
    pairs = ties = 0
    for j in range(cam.h):
        for i in range(cam.w):
            o64, d64, amin, amax = O.pixel_ray(cam, i, j)
            o32, d32 = O.pixel_ray32(k, i, j)
            for leaf in range(f.nleaves):
                iv64, tie = O.ray_leaf_intervals(of, leaf, o64, d64, amin, amax, band_rel=1e-6)
                iv32 = O.ray_leaf32(of, leaf, o32, d32, k.amin, k.amax, tabs)
                if not iv64 and not iv32:
                    continue
                pairs += 1
                if tie:
                    ties += 1
                    continue
                assert len(iv32) == len(iv64), (name, i, j, leaf, iv32, iv64)
                for (a, b), (p, q) in zip(iv64, iv32):
                    assert abs(p - a) <= 32 * EPS32 * max(abs(a), 1.0), (name, i, j, leaf)
                    assert abs(q - b) <= 32 * EPS32 * max(abs(b), 1.0), (name, i, j, leaf)
                if iv32:
                    r = rect[leaf]
                    assert r[0] <= i <= r[1] and r[2] <= j <= r[3], (name, i, j, leaf)
    assert pairs > 50 and ties <= 0.01 * pairs


def test_images_with_fp32_decisions_match_the_fp64_definition(case):
    """The whole image rendered with the FP32 decisions against the all-FP64
    oracle: pixels within 1e-5 (the FP32 rays and end points move the values
    by a few 1e-7), segment counts equal on every ray off the FP64 tie band."""
    name, f, tf, cam = case
    integ = {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}
    a = O.render(f, tf, cam, integ, bg=(0.1, 0.2, 0.3))
    b = O.render(f, tf, cam, integ, bg=(0.1, 0.2, 0.3), decide32=False, band_rel=1e-6)
    assert np.abs(a["rgba"] - b["rgba"]).max() <= 1e-5
    assert not ((a["counts"] != b["counts"]) & ~b["uncertain"]).any()
    assert not a["uncertain"].any()
    assert a["segments"] > 0
