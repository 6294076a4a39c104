"""GB300 (sm_103a) binned harmonic 3PCF estimator of arXiv:2408.16847.

The numerical path lives in libtpcf.so (C ABI: include/tpcf.h, CUDA sources in
csrc/).  ``tpcf`` is the thin PyTorch-facing wrapper; ``build`` compiles the
library in-tree.
"""
import importlib

from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("tpcf", "Plan", "ZetaFn", "Batch"):
        mod = importlib.import_module(__name__ + ".tpcf")
        return mod if name == "tpcf" else getattr(mod, name)
    raise AttributeError(name)
