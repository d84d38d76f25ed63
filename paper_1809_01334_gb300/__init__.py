"""GB300-native forest-of-octrees raycaster (Burstedde 2018, arXiv:1809.01334).

The render path -- pruning of octree leaves, per-leaf ray segments, and
order-aware aggregation of each ray's segments up the octree -- runs in the
hand-written CUDA library under ``csrc/`` behind the C ABI of
``include/ocraycast.h``.  ``capi`` marshals arguments to it; ``Renderer``
holds the device tensors (PyTorch supplies device memory and streams only).
``inputs`` builds the seeded synthetic forests, fields, transfer functions
and cameras.
"""
from __future__ import annotations

__all__ = ["Renderer", "RenderFunction", "capi", "inputs"]


def __getattr__(name):
    if name in ("Renderer", "RenderFunction"):
        from . import renderer
        return getattr(renderer, name)
    if name in ("capi", "inputs"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
