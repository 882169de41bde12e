"""GB300 (sm_103a) 2D Gaussian Splatting feature rasterizer with Precise
Tile Intersection and Top-K Hard Selection (Fast-SegSim, arXiv 2604.10951).

The compute path is ``libfss.so`` (CUDA kernels behind the C ABI in
``include/fss.h``); ``raster`` wraps it for torch tensors and autograd.
"""
from . import scenes  # noqa: F401  (pure numpy, always importable)

__all__ = ["scenes", "build", "raster"]


def build(force: bool = False) -> str:
    from .build import build as _build
    return _build(force=force)


def __getattr__(name):
    if name in ("raster", "_lib"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
