"""Parity of the CUDA shell path (cubed-sphere forests, through the C ABI) with
the FP64 oracle: images within 1e-4 per RGBA channel, visible-leaf sets,
pixel rectangles and per-ray segment counts bit-exact on every leaf and ray
(both sides decide them in FP32 by the same canonical evaluation).
"""
import numpy as np
import pytest
import torch

from paper_1809_01334_gb300 import inputs as I
from tests.test_gpu_parity import _compare

pytestmark = pytest.mark.gpu

DOPRI_C3 = {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16}


def _uniform_shell(level, kappa_max=20.0):
    f = I.shell_forest(I.shell_noise(1809, 8), level, level, 1e9)
    tf = I.transfer_function(f.nodal, 1334, kappa_max=kappa_max)
    return f, tf


def test_small_adaptive_shell_dopri5():
    """Adaptive unbalanced shell (levels 1..3, 1,518 leaves), 40x32
    perspective, DOPRI5 tol 1e-5 inside Algorithm 1 (the C3 integrator)."""
    f, tf, cam = I.preset_shell_small()
    err, st, ref = _compare(f, tf, cam, DOPRI_C3)
    assert st["segments"] > 0 and (ref["counts"] >= 2).mean() > 0.3


@pytest.mark.parametrize("method", ["rk4", "gauss2", "simpson", "equilibrium"])
def test_uniform_shell_integrators(method):
    """Uniform level-2 shell (384 leaves) with every integrator and a
    background."""
    f, tf = _uniform_shell(2)
    cam = I.perspective_camera(5, 33, 27, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    integ = {"rk4": {"method": "rk4", "nsteps": 4},
             "gauss2": {"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
             "simpson": {"method": "simpson", "c_rk": 0.2, "max_depth": 16},
             "equilibrium": {"method": "equilibrium", "c_rk": 0.2, "max_depth": 16}}[method]
    _compare(f, tf, cam, integ, bg=(0.3, 0.2, 0.1))


def test_rays_through_the_hollow_give_two_segments_per_leaf():
    """Level-0 and level-1 shells seen through the centre: rays cross the
    hollow, so one leaf can hold two segments of a ray."""
    for level in (0, 1):
        f, tf = _uniform_shell(level)
        cam = I.perspective_camera(9, 24, 20, dist=(2.0, 2.2), target=(0.0, 0.0, 0.0))
        err, st, ref = _compare(f, tf, cam, {"method": "rk4", "nsteps": 8})
        if level == 0:
            assert ref["counts"].max() >= 2


def test_cameras_inside_the_shell():
    """The eye in the hollow (every ray leaves through the shell) and in the
    shell material (the near plane clips leaves around the eye)."""
    f, tf, _ = I.preset_shell_small()
    for o, target in [((0.05, -0.02, 0.03), (1.0, 0.3, 0.2)), ((0.0, 0.78, 0.1), (0.0, 0.0, 0.0))]:
        o = np.asarray(o)
        v = np.asarray(target) - o
        v = v / np.linalg.norm(v)
        up = np.array([0.0, 0.0, 1.0])
        t = np.cross(v, up)
        t /= np.linalg.norm(t)
        u = np.cross(t, v)
        w, h, near = 30, 24, float(np.float32(0.05))
        ell = 2 * near * np.tan(np.radians(35.0)) / h
        cam = I.Camera(o=tuple(I._f32(o)), v=tuple(I._f32(v * near)), t=tuple(I._f32(t)),
                       u=tuple(I._f32(u)), ell=float(np.float32(ell)), near=near, far=50.0,
                       w=w, h=h)
        err, st, ref = _compare(f, tf, cam, DOPRI_C3)
        assert (ref["counts"] > 0).all()


@pytest.mark.parametrize("wh", [(1, 1), (37, 23), (64, 1)])
def test_ragged_images(wh):
    f, tf, _ = I.preset_shell_small()
    cam = I.perspective_camera(7, wh[0], wh[1], dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    _compare(f, tf, cam, DOPRI_C3)


def test_shell_batch_equals_single_renders():
    """Two cameras in one call (internal streams, CUDA graph capturable)
    give the same pixels as two single-camera renders."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, cam = I.preset_shell_small()
    cam2 = I.perspective_camera(11, 20, 30, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    r = Renderer(f, tf, DOPRI_C3)
    singles = []
    for c in (cam, cam2):
        r.set_camera(c)
        img, _ = r.render()
        singles.append(img.clone())
    r.set_cameras([cam, cam2])
    out, views, _ = r.render_batch()
    g = torch.cuda.CUDAGraph()
    out2 = torch.empty_like(out)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.render_batch(out=out2, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        r.render_batch(out=out2)
    out2.zero_()
    g.replay()
    torch.cuda.synchronize()
    for v, sgl in zip(views, singles):
        assert torch.equal(v, sgl)
    assert torch.equal(out, out2)
    r.close()


def test_c3_full_size_sampled_rows():
    """C3 at full size: 5,001,233 leaves (levels 4..7), 2048x2048, DOPRI5
    tol 1e-5: whole-image render on the GPU, 128 rows spread over the whole
    image against the oracle -- every pixel within the image tolerance and
    every ray's segment count (about 100 per ray) equal."""
    f, tf, cam, integ = I.preset_c3()
    assert f.nleaves == 5_001_233
    rows = np.linspace(0, cam.h - 1, 128).astype(int)
    err, st, ref = _compare(f, tf, cam, integ, rows=rows)
    assert st["segments"] > 1e8


def test_shell_empty_view_is_background():
    """A camera looking away from the shell: no leaf survives pruning, every
    pixel is the background with alpha 0."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_shell_small()
    cam = I.Camera(o=(0.0, 0.0, 3.0), v=(0.0, 0.0, 0.1), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                   ell=float(np.float32(1e-3)), near=float(np.float32(0.1)), far=100.0, w=17, h=9)
    bg = (0.25, 0.5, 0.75)
    r = Renderer(f, tf, DOPRI_C3, bg=bg)
    r.set_camera(cam)
    img, st = r.render(with_index=True)
    torch.cuda.synchronize()
    assert st["visible_leaves"] == 0 and st["segments"] == 0
    exp = torch.tensor([bg[0], bg[1], bg[2], 0.0], device=img.device).expand_as(img)
    assert torch.equal(img, exp)
    r.close()
