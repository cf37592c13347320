"""GB300-native (sm_103a) real-time signed distance fields for soft shadows.

Implements "RTSDF: Generating Signed Distance Fields in Real Time for Soft
Shadow Rendering" (Tan, Chua, Koh, Bhojan, PG 2020) as hand-written CUDA
kernels behind the C ABI of ``include/rtsdf.h`` (``librtsdf.so``):

* Sec. 2.1 -- conservative voxelization and 3D jump flooding (coarse SDF);
* Sec. 2.2 -- near-surface Philox ray tracing against a BVH with the Eq. 1
  temporal minimum and the front/back sign vote (fine SDF);
* Sec. 2.3 -- sphere-traced soft shadows and their adjoint.

The library must be built (``build.build()``); there is no CPU fallback.
"""
from ._abi import RtsdfError, STATUS_NAMES  # noqa: F401
from .context import RTSDF, RTSDFBatch  # noqa: F401

__all__ = ["RTSDF", "RTSDFBatch", "RtsdfError", "soft_shadow", "ShadowFn"]


def __getattr__(name):
    if name in ("soft_shadow", "ShadowFn"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
