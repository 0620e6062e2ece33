"""GB300-native hierarchical state-vector simulator (arXiv 2205.06973).

The compute path is ``libhisvsim.so`` (C ABI in ``include/hisvsim.h``, CUDA
kernels for sm_103a in ``csrc/``); ``_native`` binds it with ctypes and
``api`` wraps the handles around torch-owned device memory. Submodules are
imported lazily so that building the library does not need it loaded.
"""
import importlib

__all__ = ["api", "build"]


def __getattr__(name):
    if name in ("api", "build", "batch", "serving", "autotune"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
