"""GB300 decode path for the Group codecs of arXiv 1502.01916.

The compute lives in ``libgc.so`` (hand-written CUDA for sm_103a, C ABI
declared in ``include/gc.h``). This package is the thin Python binding over
that ABI: it marshals torch tensors (device memory and streams) into the C
calls, which keep the C names (``gc_encode``, ``gc_decode``,
``gc_decode_batch`` ...). There is no CPU fallback: importing the binding
without the built library raises.
"""
from .gc import *  # noqa: F401,F403
from .gc import __all__  # noqa: F401
