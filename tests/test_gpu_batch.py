"""Several cameras in one render call (the paper's multiple image instances,
Sec. 3): each camera's image is bit-identical to its own single-camera
render, one of them matches the FP64 oracle, and the batch can be captured in
a CUDA graph and replayed with new data."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_01334_gb300 import inputs as I

pytestmark = pytest.mark.gpu

INTEG = {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}


def _cams():
    return [I.perspective_camera(31, 40, 30), I.perspective_camera(32, 17, 57),
            I.perspective_camera(33, 64, 64), I.perspective_camera(34, 1, 9)]


def test_batch_equals_single_renders_and_oracle():
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_small()
    cams = _cams()
    r = Renderer(f, tf, INTEG)
    r.set_cameras(cams)
    flat, views, st = r.render_batch(with_index=True)
    torch.cuda.synchronize()
    total = 0
    vis_union = np.zeros(f.nleaves, bool)
    for cam, v in zip(cams, views):
        s = Renderer(f, tf, INTEG)
        s.set_camera(cam)
        img, st1 = s.render(with_index=True)
        torch.cuda.synchronize()
        assert torch.equal(img, v)
        total += st1["segments"]
        vis_union |= st1["visible"].cpu().numpy().astype(bool)
        s.close()
    assert st["segments"] == total
    np.testing.assert_array_equal(st["visible"].cpu().numpy().astype(bool), vis_union)
    ref = O.render(f, tf, cams[2], INTEG)
    assert np.abs(views[2].cpu().numpy() - ref["rgba"]).max() <= 1e-4
    r.close()


@pytest.mark.parametrize("merge", [0, 1])  # 0: the persistent kernel; 1: kernel chains on streams
def test_batch_in_a_cuda_graph(merge):
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_small()
    r = Renderer(f, tf, INTEG)
    r.set_cameras(_cams())
    r.set_tuning(merge=merge, persistent=1)
    nodal = r.nodal.clone()
    r.set_data(nodal, r.tf)
    out = torch.empty((r.batch_pixels(), 4), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.render_batch(out, stream=s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.render_batch(out, stream=torch.cuda.current_stream())
    for scale in (1.0, 1.03):
        nodal.copy_(r.nodal * 0 + torch.from_numpy(f.nodal).cuda() * scale)
        g.replay()
        torch.cuda.synchronize()
        ref, _, _ = r.render_batch()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    r.close()


@pytest.mark.parametrize("merge", [0, 1])
@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_every_tile_depth_matches_the_oracle(depth, merge):
    """The autotuner's tile depths (octree levels merged inside one CTA) and
    both merges of the levels above (per-level passes, one top-down pass) all
    give the oracle's images and segment counts, on several cameras at once
    with 1, 2 and 8 internal streams."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_small()
    cams = _cams()
    r = Renderer(f, tf, INTEG)
    r.set_cameras(cams)
    for streams in (1, 2, 8):
        r.set_tuning(tile_depth=depth, streams=streams, merge=merge)
        assert r.get_tuning()["tile_depth"] == depth
        flat, views, st = r.render_batch(with_index=True)
        torch.cuda.synchronize()
        for k in (0, 2):
            ref = O.render(f, tf, cams[k], INTEG)
            assert np.abs(views[k].cpu().numpy() - ref["rgba"]).max() <= 1e-4
            at = sum(c.w * c.h for c in cams[:k])
            cnt = st["counts"][at:at + cams[k].w * cams[k].h].cpu().numpy().reshape(ref["counts"].shape)
            np.testing.assert_array_equal(cnt, ref["counts"])
    r.close()


@pytest.mark.parametrize("kind", ["cube", "shell"])
def test_autotune_keeps_the_fastest_valid_setting(kind):
    from paper_1809_01334_gb300 import Renderer
    if kind == "cube":
        f, tf, _ = I.preset_small()
        cams = _cams()
    else:
        f, tf, _ = I.preset_shell_small()
        cams = [I.perspective_camera(41 + k, 24 + 7 * k, 20, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
                for k in range(3)]
    r = Renderer(f, tf, INTEG)
    r.set_cameras(cams)
    res = r.autotune(reps=2)
    tried, best = res["tried"], res["best"]
    assert len(tried) >= 4 and all(t["ms"] > 0 for t in tried)
    assert best["ms"] == min(t["ms"] for t in tried)
    assert r.get_tuning() == {**best, "ms": 0.0}
    flat, views, st = r.render_batch()
    torch.cuda.synchronize()
    ref = O.render(f, tf, cams[1], INTEG)
    assert np.abs(views[1].cpu().numpy() - ref["rgba"]).max() <= 1e-4
    r.close()


@pytest.mark.parametrize("kind", ["cube", "shell"])
def test_render_view_equals_the_batch(kind):
    """ocr_render_view renders one planned camera of a batch alone: the same
    pixels and segment counts as that camera's part of the batch render, for
    every view, in any order; a view out of range is rejected."""
    from paper_1809_01334_gb300 import Renderer, capi
    if kind == "cube":
        f, tf, _ = I.preset_small()
        cams = _cams()
    else:
        f, tf, _ = I.preset_shell_small()
        cams = [I.perspective_camera(41 + k, 24 + 7 * k, 20, dist=(2.2, 2.6), target=(0.0, 0.0, 0.0))
                for k in range(3)]
    r = Renderer(f, tf, INTEG)
    r.set_cameras(cams)
    flat, views, st = r.render_batch(with_index=True)
    torch.cuda.synchronize()
    at = 0
    starts = []
    for c in cams:
        starts.append(at)
        at += c.w * c.h
    for k in reversed(range(len(cams))):
        img, s1 = r.render_view(k, with_counts=True)
        torch.cuda.synchronize()
        assert torch.equal(img, views[k])
        cnt = st["counts"][starts[k]:starts[k] + cams[k].w * cams[k].h].view(cams[k].h, cams[k].w)
        assert torch.equal(s1["counts"], cnt)
        assert s1["segments"] == int(cnt.sum())
    with pytest.raises(capi.OcrError) as e:
        capi.render_view(r.h, len(cams), views[0])
    assert e.value.code == capi.ERR_INVALID
    r.close()


@pytest.mark.parametrize("chunks,ctas", [(1, 0), (2, 4), (16, 0), (3, 7), (32, 6)])
def test_persistent_kernel_equals_the_stream_path(chunks, ctas):
    """The persistent multi-camera kernel (one launch drawing every camera's
    pruning, prefix-sum, subtree, coarsening and pixel items from one queue)
    gives the per-camera kernel chains' pixels and counts bit for bit, for
    several ticket sizes and occupancies, at every tile depth."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, _ = I.preset_small()
    cams = _cams() + [I.perspective_camera(35, 23, 31), I.perspective_camera(36, 70, 5)]
    r = Renderer(f, tf, INTEG)
    r.set_cameras(cams)
    for depth in (1, 2, 3, 4):
        r.set_tuning(tile_depth=depth, streams=2, persistent=0, merge=0)
        ref, _, sref = r.render_batch(with_index=True)
        ref = ref.clone()
        r.set_tuning(tile_depth=depth, streams=2, persistent=1, merge=0, chunks_per_item=chunks,
                     ctas_per_sm=ctas)
        out, _, st = r.render_batch(with_index=True)
        torch.cuda.synchronize()
        assert st["launches"] == 1
        assert torch.equal(out, ref)
        assert torch.equal(st["counts"], sref["counts"])
        assert torch.equal(st["visible"], sref["visible"])
        assert st["segments"] == sref["segments"] and st["rk_steps"] == sref["rk_steps"]
    r.close()


def test_persistent_batch_of_the_large_forest_against_the_oracle():
    """The batching workload's forest (2,053,451 leaves, DOPRI5 tol 1e-6) with
    six seeded cameras of uneven square sizes in one persistent launch: every
    pixel of every camera within 1e-4 of the oracle, every ray's segment count
    equal."""
    from paper_1809_01334_gb300 import Renderer
    f, tf, _, integ = I.preset_c2(w=8, h=8)
    cams = I.batch_cameras(6, lo=48, ratio=4.0)
    r = Renderer(f, tf, integ)
    r.set_cameras(cams)
    r.set_tuning(merge=0, persistent=1)  # the persistent kernel
    assert r.get_tuning()["persistent"] == 1
    flat, views, st = r.render_batch(with_index=True)
    torch.cuda.synchronize()
    assert st["launches"] == 1
    at = 0
    for cam, v in zip(cams, views):
        ref = O.render(f, tf, cam, integ)
        assert np.abs(v.cpu().numpy() - ref["rgba"]).max() <= 1e-4
        cnt = st["counts"][at:at + cam.w * cam.h].cpu().numpy().reshape(ref["counts"].shape)
        np.testing.assert_array_equal(cnt, ref["counts"])
        at += cam.w * cam.h
    r.close()
