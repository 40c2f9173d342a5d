"""cootgb -- fused evaluation of Armadillo-style matrix expression trees on one GB300.

The public API (``Mat``, ``trans``, ``exp``, ``accu``, ``sum``, ... and
``evaluate``) lives in :mod:`paper_2508_11385_gb300.expr` and is loaded lazily
so that the seeded input generators in :mod:`paper_2508_11385_gb300.workloads`
import without the compiled library.  Every other attribute needs the CUDA
library ``libcootgb.so`` and raises if it has not been built.
"""

__all__ = ["expr", "workloads"]


def __getattr__(name):
    import importlib

    if name in ("workloads", "expr", "lib", "autograd", "build", "cube"):
        return importlib.import_module("." + name, __name__)
    if name in ("Cube", "cube_empty", "each_slice"):
        return getattr(importlib.import_module(".cube", __name__), name)
    mod = importlib.import_module(".expr", __name__)
    return getattr(mod, name)
