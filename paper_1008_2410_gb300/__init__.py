"""GB300 (sm_103a) library for one Fast Multipole velocity evaluation of 2D Gaussian vortex blobs
(M. G. Knepley, "Removing the Barrier to Scalability in Parallel FMM").

``FMM`` (handle over the C ABI of ``include/fmm2d.h``) and ``fmm_velocity`` (differentiable, with the
library's adjoint) are loaded lazily, so ``build`` and ``model`` import without torch or a GPU.
"""
from __future__ import annotations

__all__ = ["FMM", "FMMVelocity", "fmm_velocity", "build", "model"]


def __getattr__(name):
    if name in ("FMM", "FMMVelocity", "fmm_velocity"):
        from . import api

        return getattr(api, name)
    if name in ("build", "model"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
