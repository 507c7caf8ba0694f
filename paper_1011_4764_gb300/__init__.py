"""GB300-native hot path of the overlapping fragments method (OFM).

The compute lives in libofm.so (CUDA kernels for sm_103a behind the C ABI in
include/ofm.h); ``ofm`` is its thin ctypes binding and ``build`` compiles it
in-tree.
"""
from . import build  # noqa: F401


def context(stream=None):
    """A library context on the current CUDA device (loads libofm.so)."""
    from .ofm import Context
    return Context(stream)
