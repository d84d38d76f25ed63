"""The CUDA adjoint on cubed-sphere shell forests (27 nodal values per leaf)
against the FP64 oracle gradient and central differences of the FP64 forward
oracle: relative L2 error of the gradient vectors <= 1e-3; per coordinate,
error relative to max(|g_ref|, 1e-3 max|g_ref|) <= 1e-3 (tests/gradcheck.py:
with the oracle's allowances for cancelling sums and adaptive step trees, on
every coordinate).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import inputs as I
from tests import gradcheck

pytestmark = pytest.mark.gpu

DOPRI = {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5, "max_depth": 16}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("integ", [{"method": "rk4", "nsteps": 4}, DOPRI,
                                   {"method": "gauss2", "c_rk": 0.05, "max_depth": 16},
                                   {"method": "simpson", "c_rk": 0.2, "max_depth": 16},
                                   {"method": "equilibrium", "c_rk": 0.2, "max_depth": 16}])
def test_shell_gradient_matches_oracle(integ):
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_shell_small()
    cam = I.perspective_camera(21, 24, 18, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    bg = (0.1, 0.05, 0.2)
    r = Renderer(f, tf, integ, bg=bg)
    r.set_camera(cam)
    W = np.random.default_rng(3).uniform(-1, 1, (cam.h, cam.w, 4)).astype(np.float32)
    gn, gt = r.backward(torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    assert gn.shape == (f.nleaves, 27)
    rn, rt, an, at = O.render_grad(f, tf, cam, integ, W.astype(np.float64), bg=bg,
                                   magnitudes=True)
    en = _rel(gn.cpu().numpy().astype(np.float64), rn)
    et = _rel(gt.cpu().numpy().astype(np.float64), rt)
    assert en <= 1e-3 and et <= 1e-3, (en, et)
    adaptive = integ["method"] != "rk4"  # Algorithm 1: step trees in FP32 and FP64
    gradcheck.check(gn.cpu().numpy(), rn, "nodal", None if adaptive else an, max_frac=1e-3,
                    abs_frac=1e-3 if adaptive else 1e-4)
    gradcheck.check(gt.cpu().numpy(), rt, "knots", None if adaptive else at, max_frac=0.1,
                    abs_frac=1e-3 if adaptive else 1e-4)
    r.close()


def test_shell_autograd_l2_loss_against_perturbed_target():
    """The configuration of the differentiation workload at small size: L2
    loss against a target rendered from a seeded 5% perturbation of the nodal
    values, gradients through RenderFunction, against the oracle gradient and
    central differences on 64 coordinates (48 nodal values of visible leaves,
    16 knot values)."""
    from paper_1809_01334_gb300 import Renderer, RenderFunction
    f, tf, _ = I.preset_shell_small()
    cam = I.perspective_camera(23, 20, 16, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    r = Renderer(f, tf, DOPRI)
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
    gn = nodal.grad.cpu().numpy().astype(np.float64)
    gt = knots.grad.cpu().numpy().astype(np.float64)
    W = (2.0 * (img - target)).detach().cpu().numpy().astype(np.float64)
    rn, rt = O.render_grad(f, tf, cam, DOPRI, W)
    assert _rel(gn, rn) <= 1e-3 and _rel(gt, rt) <= 1e-3
    vis = O.cull(f, tf, cam)["visible"]
    cand = np.flatnonzero(np.repeat(vis, 27) & (np.abs(rn.reshape(-1)) > 0))
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
        a = O.render(f, tf, cam, DOPRI)
        arr[k] = vm
        b = O.render(f, tf, cam, DOPRI)
        arr[k] = np.float32(v)
        if a["steps"] != b["steps"]:
            continue  # the perturbation changed the adaptive step tree
        fd = float(((a["rgba"] - b["rgba"]) * W).sum()) / (float(vp) - float(vm))
        g = gn.reshape(-1)[k] if kind == "n" else gt.reshape(-1)[k]
        assert abs(g - fd) <= 1e-3 * max(abs(fd), 1e-3 * gmax), (kind, k, g, fd)
        checked += 1
    assert checked >= 56
    r.close()


def test_c5_full_size_gradient_on_sampled_rows():
    """The differentiation workload at full size (shell levels 4..6, 1024x1024,
    DOPRI5 tol 1e-5): the GPU adjoint of the L2 loss against the perturbed
    target, restricted to 32 image rows spread over the image, against the
    FP64 oracle gradient of the same restricted loss: the vector norms and
    every coordinate."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, cam, integ = I.preset_c5()
    r = Renderer(f, tf, integ)
    r.set_camera(cam)
    rng = np.random.default_rng(1809)
    pert = (f.nodal * (1 + 0.05 * rng.uniform(-1, 1, f.nodal.shape))).astype(np.float32)
    base = r.nodal.clone()
    r.set_data(torch.from_numpy(pert).cuda(), r.tf.clone())
    target, _ = r.render()
    target = target.clone()
    r.set_data(base, r.tf)
    img, _ = r.render()
    rows = np.linspace(0, cam.h - 1, 32).astype(int).tolist()
    W = torch.zeros_like(img)
    W[rows] = 2.0 * (img[rows] - target[rows])
    gn, gt = r.backward(W)
    torch.cuda.synchronize()
    Wn = W.cpu().numpy().astype(np.float64)
    rn, rt = O.render_grad(f, tf, cam, integ, Wn)
    assert np.abs(rn).max() > 0
    en = _rel(gn.cpu().numpy().astype(np.float64), rn)
    et = _rel(gt.cpu().numpy().astype(np.float64), rt)
    assert en <= 1e-3 and et <= 1e-3, (en, et)
    # DOPRI5 step trees taken in FP32 and FP64 differ near their thresholds: on
    # a few coordinates dominated by such a segment the two gradients differ
    # by up to about 1e-3 of the largest entry (tests/gradcheck.py)
    gradcheck.check(gn.cpu().numpy(), rn, "nodal", max_frac=1e-4, abs_frac=2e-3)
    gradcheck.check(gt.cpu().numpy(), rt, "knots", max_frac=0.1, abs_frac=2e-3)
    r.close()


def test_shell_backward_is_graph_capturable():
    """The shell adjoint enqueues its work without waiting (its list sizes
    come from the camera's plan): captured in a CUDA graph, its replays give
    the gradient of a direct call (atomic sums: equal up to their order)."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_shell_small()
    cam = I.perspective_camera(21, 40, 30, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
    r = Renderer(f, tf, DOPRI)
    r.set_camera(cam)
    W = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, (cam.h, cam.w, 4))
                         .astype(np.float32)).cuda()
    gn, gt = r.backward(W)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.backward(W, check=False)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gn_c, gt_c = r.backward(W, check=False)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    r.sync()
    for a, b in ((gn.cpu().numpy(), gn_c.cpu().numpy()), (gt.cpu().numpy(), gt_c.cpu().numpy())):
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30)
    r.close()
