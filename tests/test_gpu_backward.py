"""The CUDA adjoint (ocr_render_backward) against the FP64 oracle gradient and
against central differences of the FP64 forward oracle.

Targets: relative L2 error of the full gradient vectors <= 1e-3; on 64
coordinates (48 nodal values of visible leaves, 16 knot values) the error
relative to max(|g_ref|, 1e-3 max|g_ref|) <= 1e-3; every coordinate against
the oracle gradient by tests/gradcheck.py (the same strict test, with the
oracle's allowances for cancelling sums and adaptive step trees).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import inputs as I
from tests import gradcheck

pytestmark = pytest.mark.gpu


def _setup(kind, integ, w=24, h=18):
    if kind == "uniform2":
        f = I.uniform_cube_forest(2, I.gaussian_field(4, 1809))
    else:
        f = I.adaptive_cube_forest(I.gaussian_field(16, 99), 1, 4, 0.3, balance=True)
    tf = I.transfer_function(f.nodal, 1334, kappa_max=12.0)
    cam = I.perspective_camera(21, w, h, dist=(1.7, 2.1))
    return f, tf, cam


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("kind", ["uniform2", "adaptive"])
@pytest.mark.parametrize("integ", [{"method": "rk4", "nsteps": 4},
                                   {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16},
                                   {"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
                                   {"method": "simpson", "c_rk": 0.2, "max_depth": 16},
                                   {"method": "equilibrium", "c_rk": 0.2, "max_depth": 16}])
def test_gradient_matches_oracle(kind, integ):
    from paper_1809_01334_gb300 import Renderer
    f, tf, cam = _setup(kind, integ)
    bg = (0.1, 0.05, 0.2)
    r = Renderer(f, tf, integ, bg=bg)
    r.set_camera(cam)
    W = np.random.default_rng(3).uniform(-1, 1, (cam.h, cam.w, 4)).astype(np.float32)
    gn, gt = r.backward(torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    rn, rt, an, at = O.render_grad(f, tf, cam, integ, W.astype(np.float64), bg=bg,
                                   magnitudes=True)
    en, et = _rel(gn.cpu().numpy().astype(np.float64), rn), _rel(gt.cpu().numpy().astype(np.float64), rt)
    assert en <= 1e-3 and et <= 1e-3, (en, et)
    adaptive = integ["method"] != "rk4"  # Algorithm 1: step trees in FP32 and FP64
    gradcheck.check(gn.cpu().numpy(), rn, "nodal", None if adaptive else an, max_frac=1e-2,
                    abs_frac=1e-3 if adaptive else 1e-4)
    gradcheck.check(gt.cpu().numpy(), rt, "knots", None if adaptive else at, max_frac=0.1,
                    abs_frac=1e-3 if adaptive else 1e-4)
    r.close()


def test_autograd_l2_loss_against_perturbed_target():
    """Sec. 2 differentiated end to end: L2 loss between the image and a target
    rendered from a seeded 5% perturbation of the nodal values; gradients via
    torch.autograd through RenderFunction, compared with the oracle gradient of
    the same loss and with central differences on 64 coordinates."""
    from paper_1809_01334_gb300 import Renderer, RenderFunction
    integ = {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}
    f, tf, cam = _setup("adaptive", integ, w=20, h=16)
    r = Renderer(f, tf, integ)
    r.set_camera(cam)
    rng = np.random.default_rng(5)
    pert = (f.nodal * (1 + 0.05 * rng.uniform(-1, 1, f.nodal.shape))).astype(np.float32)
    r.set_data(torch.from_numpy(pert).cuda(), r.tf.clone())
    target, _ = r.render()
    target = target.clone()
    nodal = torch.from_numpy(f.nodal.copy()).cuda().requires_grad_(True)
    knots = torch.from_numpy(tf.knots.copy()).cuda().requires_grad_(True)
    img = RenderFunction.apply(nodal, knots, r)
    loss = ((img - target) ** 2).sum()
    loss.backward()
    gn, gt = nodal.grad.cpu().numpy().astype(np.float64), knots.grad.cpu().numpy().astype(np.float64)
    W = (2.0 * (img - target)).detach().cpu().numpy().astype(np.float64)
    rn, rt = O.render_grad(f, tf, cam, integ, W)
    assert _rel(gn, rn) <= 1e-3 and _rel(gt, rt) <= 1e-3
    # central differences of the FP64 oracle on 64 coordinates (linearised loss)
    vis = O.cull(f, tf, cam)["visible"]
    cand = np.flatnonzero(np.repeat(vis, 8))
    coords = [("n", int(k)) for k in rng.choice(cand, 48, replace=False)]
    coords += [("t", int(k)) for k in rng.choice(32, 16, replace=False)]
    gmax = max(np.abs(rn).max(), np.abs(rt).max())
    checked = 0
    for kind, k in coords:
        arr = f.nodal.reshape(-1) if kind == "n" else tf.knots.reshape(-1)
        v = float(arr[k])
        hh = 1e-4 * max(1.0, abs(v))
        vp, vm = np.float32(v + hh), np.float32(v - hh)
        arr[k] = vp
        a = O.render(f, tf, cam, integ)
        arr[k] = vm
        b = O.render(f, tf, cam, integ)
        arr[k] = np.float32(v)
        if a["steps"] != b["steps"]:
            continue  # the perturbation changed the adaptive step tree
        fd = float(((a["rgba"] - b["rgba"]) * W).sum()) / (float(vp) - float(vm))
        g = gn.reshape(-1)[k] if kind == "n" else gt.reshape(-1)[k]
        assert abs(g - fd) <= 1e-3 * max(abs(fd), 1e-3 * gmax), (kind, k, g, fd)
        checked += 1
    assert checked >= 56
    r.close()


def _diagonal_camera(w, h, fov_deg=12.0):
    """Perspective camera on the cube's main diagonal, looking at its centre:
    central rays cross about 3 x 2^L cells of a uniform level-L forest."""
    d = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
    o = np.array([0.5, 0.5, 0.5]) + 1.6 * d + np.array([0.013, -0.007, 0.004])
    v = -d
    up = np.array([0.0, 0.0, 1.0])
    t = np.cross(v, up)
    t /= np.linalg.norm(t)
    u = np.cross(t, v)
    near = float(np.float32(0.1))
    ell = 2 * near * np.tan(np.radians(fov_deg / 2)) / h
    return I.Camera(o=tuple(I._f32(o)), v=tuple(I._f32(v * near)), t=tuple(I._f32(t)),
                    u=tuple(I._f32(u)), ell=float(np.float32(ell)), near=near, far=100.0,
                    w=w, h=h)


def test_long_rays_gradient():
    """Rays with more than 256 segments (uniform level-7 cube seen along its
    diagonal): the per-ray scans take their shared-memory sort; the gradient
    of a loss on four rows against the oracle gradient."""
    from paper_1809_01334_gb300 import Renderer
    f = I.uniform_cube_forest(7, I.gaussian_field(4, 1809))
    tf = I.transfer_function(f.nodal, 1334, kappa_max=3.0)
    cam = _diagonal_camera(48, 36)
    integ = {"method": "rk4", "nsteps": 2}
    r = Renderer(f, tf, integ)
    r.set_camera(cam)
    _, st = r.render(with_index=True)
    counts = st["counts"].cpu().numpy() if hasattr(st["counts"], "cpu") else np.asarray(st["counts"])
    rows = [16, 17, 18, 19]
    assert counts.reshape(cam.h, cam.w)[rows].max() > 256
    W = np.zeros((cam.h, cam.w, 4), np.float32)
    W[rows] = np.random.default_rng(11).uniform(-1, 1, (len(rows), cam.w, 4))
    gn, gt = r.backward(torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    rn, rt, an, at = O.render_grad(f, tf, cam, integ, W.astype(np.float64), magnitudes=True)
    en, et = _rel(gn.cpu().numpy().astype(np.float64), rn), _rel(gt.cpu().numpy().astype(np.float64), rt)
    assert en <= 1e-3 and et <= 1e-3, (en, et)
    gradcheck.check(gn.cpu().numpy(), rn, "nodal", an)
    gradcheck.check(gt.cpu().numpy(), rt, "knots", at, max_frac=0.1)
    r.close()


@pytest.mark.parametrize("geometry", ["cube", "shell"])
def test_empty_view_gradient_is_zero(geometry):
    """A camera that sees no leaf: no pairs, no hits, no segments; the adjoint
    returns zero gradients without an error."""
    from paper_1809_01334_gb300 import Renderer
    if geometry == "cube":
        f, tf, _ = I.preset_small("adaptive")
        cam = I.Camera(o=(0.5, 0.5, 3.0), v=(0.0, 0.0, 0.1), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                       ell=float(np.float32(1e-3)), near=float(np.float32(0.1)), far=100.0,
                       w=19, h=11)
    else:
        f, tf, _ = I.preset_shell_small()
        cam = I.Camera(o=(0.0, 0.0, 3.0), v=(0.0, 0.0, 0.1), t=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                       ell=float(np.float32(1e-3)), near=float(np.float32(0.1)), far=100.0,
                       w=19, h=11)
    r = Renderer(f, tf, {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16})
    r.set_camera(cam)
    img, st = r.render(with_index=True)
    assert st["segments"] == 0
    W = torch.ones((cam.h, cam.w, 4), dtype=torch.float32, device="cuda")
    gn, gt = r.backward(W)
    torch.cuda.synchronize()
    assert float(gn.abs().max()) == 0.0 and float(gt.abs().max()) == 0.0
    r.close()


def test_backward_is_stream_ordered_and_graph_capturable():
    """After the first call for a camera (which finds the sizes of its pair
    space and hit lists), the adjoint enqueues its work without waiting: it is
    captured in a CUDA graph, and replays of the graph give the gradient of a
    direct call (atomic sums: equal up to their order); ocr_sync reports no
    device error."""
    from paper_1809_01334_gb300 import Renderer
    integ = {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}
    f, tf, cam = _setup("adaptive", integ, w=40, h=30)
    r = Renderer(f, tf, integ)
    r.set_camera(cam)
    W = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, (cam.h, cam.w, 4))
                         .astype(np.float32)).cuda()
    gn, gt = r.backward(W)  # the first call plans (blocking)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.backward(W, check=False)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gn_c, gt_c = r.backward(W, check=False)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    r.sync()
    a, b = gn.cpu().numpy(), gn_c.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30)
    a, b = gt.cpu().numpy(), gt_c.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30)
    r.close()
