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

from paper_1809_01334_gb300 import capi
from paper_1809_01334_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _geo(forest, dev):
    g = np.concatenate([forest.anchor.astype(np.int32),
                        forest.level.astype(np.int32)[:, None]], axis=1)
    return torch.from_numpy(np.ascontiguousarray(g)).to(dev)


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
