"""GB300-native engine for streaming temporal random walks (Tempest, Sec. 2).

The compute path is the CUDA library libtempest.so (C ABI in
include/tempest.h); ``_lib`` is its ctypes binding.  ``synth`` generates the
seeded synthetic edge streams used by the tests and the benchmark.
"""
from . import build  # noqa: F401

__all__ = ["build", "load", "Engine"]


def load():
    from . import _lib
    return _lib.load()


def __getattr__(name):
    if name == "Engine":
        from ._lib import Engine
        return Engine
    raise AttributeError(name)
