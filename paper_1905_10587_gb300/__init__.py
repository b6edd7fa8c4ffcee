"""GB300-native preconditioned Gaussian kernel ridge regression.

The compute path is libkrr.so (hand-written CUDA for sm_103a behind the C ABI in
include/krr.h); this package holds its build step and a thin ctypes binding.
Importing the binding requires the built library: there is no CPU fallback.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("KRR", "KRRError", "solve"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
