"""GB300-native topological charge density by symmetric multi-probing (arXiv:1901.02211).

The compute path is libsmpq.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/smpq.h); `smpq` is its ctypes binding and `session` a small
convenience layer over it.  Nothing here falls back to CPU code.
"""
from . import smpq  # noqa: F401
from .session import Session  # noqa: F401
