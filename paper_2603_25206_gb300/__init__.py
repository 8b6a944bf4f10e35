"""GB300-native multi-stage decompression and homomorphic operations (HSZ, arXiv 2603.25206).

The compute lives in libhc.so (CUDA, sm_103a, C ABI in include/hc.h); ``hc``
is its ctypes binding.  Importing the package does not load the library;
``hc.lib()`` does, and fails loudly when it has not been built.
"""
from . import hc  # noqa: F401

__all__ = ["hc"]
