"""The pruning entry point that allocates nothing (ocr_prune_noalloc).

It exists for callers that cannot allocate device memory when they need a
result -- an application serving all device memory from a pool it reserved
up front, a real-time loop that must not take the device-wide
synchronisation an allocation implies, a plug-in inside another program's
memory budget.  Its output must equal what the regular render path reports
for the same forest and camera: identical pixel rectangles, and the visible
leaves listed in Morton order.  Two calls in a row check that the shared
scratch array is reset between calls.  This file is collected last on
purpose.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import capi
from paper_1809_01334_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _geo(forest, dev, fourth=None):
    w = forest.level.astype(np.int32) if fourth is None else fourth
    g = np.concatenate([forest.anchor.astype(np.int32), w[:, None]], axis=1)
    return torch.from_numpy(np.ascontiguousarray(g)).to(dev)


def _refine_last_leaf(level):
    """A uniform forest of the given level whose last leaf (in Morton order)
    is split into its 8 children: 8^level + 7 leaves, never a multiple of the
    1024-leaf tile."""
    f = I.uniform_cube_forest(level, I.gaussian_field(4, 1809), max_level=level + 1)
    lv = f.level.astype(np.uint8).copy()
    an = f.anchor.astype(np.int32).copy()
    half = 1
    kids = np.array([[an[-1, 0] + half * (o & 1), an[-1, 1] + half * ((o >> 1) & 1),
                      an[-1, 2] + half * ((o >> 2) & 1)] for o in range(8)], np.int32)
    lv = np.concatenate([lv[:-1], np.full(8, level + 1, np.uint8)])
    an = np.concatenate([an[:-1], kids])
    lv, an, tr = I._sort_forest(lv, an, np.zeros(len(lv), np.int32))
    nodal = I._sample_corners(I.gaussian_field(4, 1809), lv, an, level + 1).astype(np.float32)
    return I.Forest("cube", level + 1, lv, an, tr, nodal, {"kind": "refined-last"})


def _x_axis_camera(w, h):
    """A narrow camera looking along +x just above the cube's y = z = 0 edge:
    only leaves touching that edge project onto pixels."""
    near = float(np.float32(0.05))
    ell = 2 * near * np.tan(np.radians(1.0)) / h
    return I.Camera(o=(-0.5, 0.02, 0.02), v=(near, 0.0, 0.0), t=(0.0, 1.0, 0.0),
                    u=(0.0, 0.0, 1.0), ell=float(np.float32(ell)), near=near, far=100.0,
                    w=w, h=h)


def _call_twice(f, cam, dev):
    geo = _geo(f, dev)
    out = []
    for call in range(2):  # the second call must not see the first one's state
        rects = torch.full((f.nleaves, 4), -7, dtype=torch.int32, device=dev)
        idx = torch.full((f.nleaves,), -7, dtype=torch.int32, device=dev)
        n = capi.prune_noalloc(geo, f.nleaves, f.max_level, cam, rects, idx,
                               stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out.append((n, rects.cpu().numpy(), idx.cpu().numpy()))
    return out


@pytest.mark.parametrize("case", ["partial_view", "uniform_level5"])
def test_prune_noalloc_matches_render(case):
    from paper_1809_01334_gb300 import Renderer
    dev = torch.device("cuda")
    if case == "partial_view":
        fld = I.gaussian_field(16, 99)
        f = I.adaptive_cube_forest(fld, 1, 5, 0.3, balance=True)
        cam = I.perspective_camera(21, 97, 61, dist=(0.9, 1.0))  # close: part of the cube
    else:
        f = I.uniform_cube_forest(5, I.gaussian_field(4, 1809))  # 32768 leaves, 32 tiles
        cam = I.perspective_camera(5, 160, 90)
    tf = I.transfer_function(f.nodal)
    r = Renderer(f, tf, {"method": "rk4", "nsteps": 2})
    r.set_camera(cam)
    _, st = r.render(with_index=True)
    torch.cuda.synchronize()
    ref_rects = st["rects"].cpu().numpy()
    ref_vis = np.nonzero(st["visible"].cpu().numpy())[0]
    assert 0 < len(ref_vis) <= f.nleaves
    if case == "partial_view":
        assert len(ref_vis) < f.nleaves
    geo = _geo(f, dev)
    for call in range(2):  # the second call must not see the first one's state
        rects = torch.full((f.nleaves, 4), -7, dtype=torch.int32, device=dev)
        idx = torch.full((f.nleaves,), -7, dtype=torch.int32, device=dev)
        n = capi.prune_noalloc(geo, f.nleaves, f.max_level, cam, rects, idx,
                               stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert n == len(ref_vis) == st["visible_leaves"], call
        np.testing.assert_array_equal(rects.cpu().numpy(), ref_rects)
        np.testing.assert_array_equal(idx[:n].cpu().numpy(), ref_vis)
    r.close()


def test_prune_noalloc_rejects_oversize():
    cam = I.perspective_camera(7, 8, 8)
    with pytest.raises(capi.OcrError) as e:
        capi.prune_noalloc(1 << 20, (1 << 26) + 1, 8, cam, None, 1 << 21)
    assert e.value.code == capi.ERR_INVALID


def test_prune_noalloc_ragged_tiles_against_the_oracle():
    """A uniform level-4 forest with its last leaf split
    (4103 leaves: five tiles, the last one holding 7 leaves), seen by a
    camera for which every visible leaf lies in the first tile: the count,
    the index list and the rectangles against the oracle's pruning."""
    dev = torch.device("cuda")
    f = _refine_last_leaf(4)
    assert f.nleaves == 4103 and f.nleaves % 1024 != 0
    tf = I.transfer_function(f.nodal)
    cam = _x_axis_camera(33, 21)
    ref = O.cull(f, tf, cam)
    vis = np.flatnonzero(ref["visible"])
    assert 0 < len(vis) and vis.max() < 1024  # all visible leaves in the first tile
    for n, rects, idx in _call_twice(f, cam, dev):
        assert n == len(vis)
        np.testing.assert_array_equal(idx[:n], vis)
        assert (idx[n:] == -7).all()  # entries past the count are untouched
        np.testing.assert_array_equal(rects[vis], ref["rect"][vis])
        assert (rects[~ref["visible"]] == [0, -1, 0, -1]).all()


def test_prune_noalloc_index_list_against_the_oracle():
    """An adaptive forest partly in view: the visible-leaf list equals the
    oracle's visible set in Morton order, and every rectangle the oracle's
    (both decide them in FP32 by the same canonical evaluation)."""
    dev = torch.device("cuda")
    f = I.adaptive_cube_forest(I.gaussian_field(16, 99), 1, 5, 0.3, balance=True)
    tf = I.transfer_function(f.nodal)
    cam = I.perspective_camera(21, 97, 61, dist=(0.9, 1.0))
    ref = O.cull(f, tf, cam)
    vis = np.flatnonzero(ref["visible"])
    assert 0 < len(vis) < f.nleaves
    for n, rects, idx in _call_twice(f, cam, dev):
        assert n == len(vis)
        np.testing.assert_array_equal(idx[:n], vis)
        np.testing.assert_array_equal(rects, ref["rect"])


def test_prune_noalloc_rejects_records_that_are_not_cube_leaves():
    """Leaf records in device memory with a level above max_level, or a
    shell record (tree in the upper bits of the fourth word): the call
    returns OCR_ERR_INVALID, and a following valid call still succeeds."""
    dev = torch.device("cuda")
    f = I.uniform_cube_forest(3, I.gaussian_field(4, 1809))
    cam = I.perspective_camera(5, 40, 30)
    rects = torch.empty((f.nleaves, 4), dtype=torch.int32, device=dev)
    idx = torch.empty((f.nleaves,), dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    for fourth, max_level in ((f.level.astype(np.int32), 2),
                              (f.level.astype(np.int32) | (3 << 8), 3)):
        geo = _geo(f, dev, fourth)
        with pytest.raises(capi.OcrError) as e:
            capi.prune_noalloc(geo, f.nleaves, max_level, cam, rects, idx, stream=st)
        assert e.value.code == capi.ERR_INVALID
    n = capi.prune_noalloc(_geo(f, dev), f.nleaves, 3, cam, rects, idx, stream=st)
    torch.cuda.synchronize()
    assert n > 0
