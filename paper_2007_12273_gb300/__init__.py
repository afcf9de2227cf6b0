"""GB300 (sm_103a) Gaussian-mixture checkpoint-restart for particle-in-cell
codes: the method of Chen, Chacon & Nguyen (arXiv 2007.12273).

``gm`` is the Python binding of the C ABI (``include/gm.h``); ``build``
compiles the CUDA library in-tree.
"""
import importlib

from . import build  # noqa: F401

__all__ = ["build", "gm"]


def __getattr__(name):
    if name == "gm":
        return importlib.import_module(__name__ + ".gm")
    raise AttributeError(name)
