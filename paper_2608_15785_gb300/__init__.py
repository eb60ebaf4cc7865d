"""GB300-native RoofGS renderer: forward render of 3D Gaussian Splatting.

The renderer is the C ABI of ``include/rg.h`` (librg.so, CUDA kernels for
sm_103a); ``binding`` marshals arguments to it. ``synth`` draws seeded
synthetic scenes and cameras. Importing this package does not load the
library; the first call that needs it does, and raises if it is missing.
"""
from . import synth  # noqa: F401
from .binding import (RG_FLAG_EXACT_EXP, RG_FLAG_SINGLE_PIXEL, RG_FLAG_SORT_FULL_KEY,  # noqa: F401
                      RG_FLAG_STAGE_EVENTS,
                      RG_MODE_EXACT, RG_MODE_ROOFGS, RG_SH_SCALE_BAND, RG_SH_SCALE_BAND_GAUSS,
                      RG_STORE_COMPACT, RG_STORE_FP32, RgError, Scene, eval_fast_exp, lib, version)


def build(force: bool = False) -> str:
    """Compile librg.so for sm_103a (nvcc) and return its path."""
    from .build import build as _build
    return _build(force=force)
