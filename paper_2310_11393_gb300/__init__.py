"""GB300 (sm_103a) scattered-field particle-in-cell hot path (arXiv 2310.11393).

The CUDA library (csrc/, built into _lib/libsffpic.so) implements the C-ABI of
include/pic.h; ``pic`` is its thin ctypes binding.
"""
from . import pic  # noqa: F401
from ._build import build  # noqa: F401
