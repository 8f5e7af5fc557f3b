"""GB300-native weighted quadrature on bicubic unstructured splines.

The compute path is the C-ABI library ``lib/libwq.so`` (hand-written CUDA for
sm_103a, include/wq.h); ``wq`` is its Python binding.
"""
from . import wq  # noqa: F401
