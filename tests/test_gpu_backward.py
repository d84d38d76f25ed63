"""The CUDA adjoint (ocr_render_backward) against the FP64 oracle gradient and
against central differences of the FP64 forward oracle.

Targets: relative L2 error of the full gradient vectors <= 1e-3; on 64
coordinates (48 nodal values of visible leaves, 16 knot values) the error
relative to max(|g_ref|, 1e-3 max|g_ref|) <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import inputs as I

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
                                   {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}])
def test_gradient_matches_oracle(kind, integ):
    from paper_1809_01334_gb300 import Renderer
    f, tf, cam = _setup(kind, integ)
    bg = (0.1, 0.05, 0.2)
    r = Renderer(f, tf, integ, bg=bg)
    r.set_camera(cam)
    W = np.random.default_rng(3).uniform(-1, 1, (cam.h, cam.w, 4)).astype(np.float32)
    gn, gt = r.backward(torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    rn, rt = O.render_grad(f, tf, cam, integ, W.astype(np.float64), bg=bg)
    en, et = _rel(gn.cpu().numpy().astype(np.float64), rn), _rel(gt.cpu().numpy().astype(np.float64), rt)
    assert en <= 1e-3 and et <= 1e-3, (en, et)
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
