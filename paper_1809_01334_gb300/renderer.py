"""Renderer: the library's handle plus the torch tensors it reads and writes."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def _stream_ptr(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Renderer:
    """Owns one ``ocr_forest`` handle.

    ``forest``: an ``inputs.Forest``; ``tf``: an ``inputs.TransferFunction``;
    ``integ``: {"method": "rk4", "nsteps": n} or {"method": "dopri5", "tol",
    "c_rk", "max_depth"}.  Nodal data and knots are copied to the device once;
    ``set_data`` replaces them (e.g. with tensors the caller updates).
    """

    def __init__(self, forest, tf, integ: dict, device="cuda", bg=(0.0, 0.0, 0.0)):
        if not torch.cuda.is_available():
            raise RuntimeError("Renderer needs a CUDA device")
        self.device = torch.device(device)
        self.forest = forest
        s = _stream_ptr(None)
        if forest.geometry == "shell":
            self.h = capi.build_forest(forest.level, forest.anchor, forest.max_level, stream=s,
                                       geometry=capi.GEOM_SHELL, tree=forest.tree,
                                       frames=forest.meta["frames"], r0=forest.meta["r0"],
                                       r1=forest.meta["r1"])
        else:
            self.h = capi.build_forest(forest.level, forest.anchor, forest.max_level, stream=s)
        self.nodal = torch.from_numpy(np.ascontiguousarray(forest.nodal, np.float32)).to(self.device)
        self.tf = torch.from_numpy(np.ascontiguousarray(tf.knots, np.float32)).to(self.device)
        self.s_min, self.s_max = float(tf.s_min), float(tf.s_max)
        capi.forest_set_data(self.h, self.nodal, self.tf, self.s_min, self.s_max, s)
        self.set_integrator(integ, bg)
        self.cam = None

    def set_data(self, nodal: torch.Tensor, tf: torch.Tensor, s_min=None, s_max=None):
        assert nodal.is_cuda and nodal.dtype == torch.float32 and nodal.is_contiguous()
        assert tf.is_cuda and tf.dtype == torch.float32 and tf.is_contiguous()
        self.nodal, self.tf = nodal, tf
        if s_min is not None:
            self.s_min, self.s_max = float(s_min), float(s_max)
        capi.forest_set_data(self.h, self.nodal, self.tf, self.s_min, self.s_max,
                             _stream_ptr(None))

    def set_integrator(self, integ: dict, bg=(0.0, 0.0, 0.0)):
        """integ["surface"] (optional): {"s_iso", "a_s", "i_s"}, the isosurface
        rendered as a surface (Sec. 2.8)."""
        surf = integ.get("surface")
        if integ["method"] == "rk4":
            capi.set_integrator(self.h, capi.RK4, nsteps=integ.get("nsteps", 4), bg=bg,
                                surface=surf)
        elif integ["method"] == "dopri5":
            capi.set_integrator(self.h, capi.DOPRI5, tol=integ.get("tol", 1e-6),
                                c_rk=integ.get("c_rk", 0.5), max_depth=integ.get("max_depth", 16),
                                bg=bg, surface=surf)
        elif integ["method"] in ("gauss2", "simpson", "equilibrium"):
            method = {"gauss2": capi.GAUSS2, "simpson": capi.SIMPSON,
                      "equilibrium": capi.EQUILIBRIUM}[integ["method"]]
            capi.set_integrator(self.h, method, c_rk=integ.get("c_rk", 0.5),
                                max_depth=integ.get("max_depth", 16), bg=bg, surface=surf)
        else:
            raise ValueError(integ["method"])

    def set_camera(self, cam):
        capi.set_camera(self.h, cam.o, cam.v, cam.t, cam.u, cam.ell, cam.near, cam.far, cam.w,
                        cam.h, cam.ortho)
        self.cam = cam
        self.cams = [cam]

    def set_cameras(self, cams):
        """Several cameras rendered together by render_batch (one call, no host
        synchronisation; capturable in a CUDA graph)."""
        capi.set_cameras(self.h, cams)
        self.cam = cams[0]
        self.cams = list(cams)

    def batch_pixels(self) -> int:
        return sum(c.w * c.h for c in self.cams)

    def render_batch(self, out: torch.Tensor | None = None, stream=None, with_index=False):
        """Render every camera into one flat buffer [sum(w*h), 4]; returns it,
        the per-camera [h, w, 4] views and the stats."""
        n = self.batch_pixels()
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        extra = {}
        if with_index:
            extra["counts"] = torch.empty(n, dtype=torch.int32, device=self.device)
            extra["visible"] = torch.empty(self.forest.nleaves, dtype=torch.uint8,
                                           device=self.device)
        st = capi.render(self.h, out, _stream_ptr(stream), d_counts=extra.get("counts"),
                         d_visible=extra.get("visible"), fill_counters=with_index)
        st.update(extra)
        views, at = [], 0
        for c in self.cams:
            views.append(out[at:at + c.w * c.h].view(c.h, c.w, 4))
            at += c.w * c.h
        return out, views, st

    def render_view(self, view: int, out: torch.Tensor | None = None, stream=None,
                    with_counts=False):
        """Render camera ``view`` of the last ``set_cameras`` alone into ``out``
        ([h, w, 4]), without planning again (ocr_render_view)."""
        cam = self.cams[view]
        if out is None:
            out = torch.empty((cam.h, cam.w, 4), dtype=torch.float32, device=self.device)
        counts = (torch.empty((cam.h, cam.w), dtype=torch.int32, device=self.device)
                  if with_counts else None)
        st = capi.render_view(self.h, view, out, _stream_ptr(stream), d_counts=counts,
                              fill_counters=with_counts)
        if with_counts:
            st["counts"] = counts
        return out, st

    def render(self, out: torch.Tensor | None = None, stream=None, with_index=False,
               fill_counters=False, time_phases=False):
        """Render into ``out`` ([h, w, 4] float32 on the device).  With
        ``with_index`` also return per-ray segment counts, per-leaf visibility
        and pixel rectangles."""
        cam = self.cam
        if out is None:
            out = torch.empty((cam.h, cam.w, 4), dtype=torch.float32, device=self.device)
        extra = {}
        if with_index:
            extra["counts"] = torch.empty((cam.h, cam.w), dtype=torch.int32, device=self.device)
            extra["visible"] = torch.empty(self.forest.nleaves, dtype=torch.uint8, device=self.device)
            extra["rects"] = torch.empty((self.forest.nleaves, 4), dtype=torch.int32,
                                         device=self.device)
        st = capi.render(self.h, out, _stream_ptr(stream), d_counts=extra.get("counts"),
                         d_visible=extra.get("visible"), d_rects=extra.get("rects"),
                         fill_counters=fill_counters or with_index, time_phases=time_phases)
        st.update(extra)
        return out, st

    def render_host(self, nodal_h: torch.Tensor, tf_h: torch.Tensor, out_h: torch.Tensor,
                    stream=None):
        """Render from host memory (ocr_render_host): ``nodal_h`` ([N, 8] or
        [N, 27]) and ``tf_h`` ([8, 4]) float32 on the host in, ``out_h`` (all
        cameras' pixels x 4 float32 on the host, e.g. [h, w, 4] for one) out;
        returns when ``out_h`` holds the image.  Afterwards the renderer's data
        is the library's device copy."""
        for t in (nodal_h, tf_h, out_h):
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("render_host takes contiguous float32 host tensors")
        if nodal_h.numel() != self.nodal.numel() or tf_h.numel() != 32:
            raise ValueError("render_host: nodal / knot sizes do not match the forest")
        if out_h.numel() != self.batch_pixels() * 4:
            raise ValueError("render_host: the image must hold 4 values per pixel of every camera")
        return capi.render_host(self.h, nodal_h, tf_h, self.s_min, self.s_max, out_h,
                                _stream_ptr(stream))

    def backward(self, grad_rgba: torch.Tensor, stream=None, check: bool = True):
        """dL/d(nodal) [N, 8] and dL/d(knots) [8, 4] (cube forests) for the data, camera and
        integrator last set, given dL/d(rgba) [h, w, 4] on the device.  The adjoint is
        stream-ordered; check=True waits for it and raises on a device error (ocr_sync),
        check=False returns at once (call sync() later)."""
        g = grad_rgba.detach().to(self.device, torch.float32).contiguous()
        gn = torch.empty_like(self.nodal)
        gt = torch.empty_like(self.tf)
        capi.render_backward(self.h, g, gn, gt, _stream_ptr(stream))
        if check:
            capi.sync(self.h, _stream_ptr(stream))
        return gn, gt

    def sync(self, stream=None):
        """Wait for the stream; raise if a stream-ordered call recorded a device error."""
        capi.sync(self.h, _stream_ptr(stream))

    def autotune(self, reps: int = 3) -> dict:
        """Time the candidate decompositions on the current cameras and keep
        the fastest (ocr_autotune)."""
        return capi.autotune(self.h, reps)

    def set_tuning(self, tile_depth: int = 4, streams: int = 4, shell_warps: int = 0,
                   merge: int = 1, persistent: int = 1, chunks_per_item: int = 16,
                   ctas_per_sm: int = 0):
        capi.set_tuning(self.h, tile_depth, streams, shell_warps, merge, persistent,
                        chunks_per_item, ctas_per_sm)

    def get_tuning(self) -> dict:
        return capi.get_tuning(self.h)

    def device_bytes(self) -> int:
        return capi.device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            capi.destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFunction(torch.autograd.Function):
    """image = render(nodal, knots) with the CUDA adjoint as its backward.

    ``RenderFunction.apply(nodal, knots, renderer)`` renders with the
    renderer's forest, camera and integrator; the backward pass calls
    ``ocr_render_backward`` (segments recomputed, not stored)."""

    @staticmethod
    def forward(ctx, nodal, knots, renderer):
        renderer.set_data(nodal.detach().contiguous(), knots.detach().contiguous())
        img, _ = renderer.render()
        ctx.renderer = renderer
        ctx.save_for_backward(nodal, knots)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        nodal, knots = ctx.saved_tensors
        r = ctx.renderer
        r.set_data(nodal.detach().contiguous(), knots.detach().contiguous())
        gn, gt = r.backward(grad_img)
        return gn, gt, None
