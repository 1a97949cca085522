"""GB300-native (sm_103a) PTHR hot path: Parallel Tempering with all-cluster
Houdayer moves and an entropic Reservoir for the 3D Edwards-Anderson spin
glass (arXiv 2605.25872).

The compute lives in libpthr.so (CUDA kernels behind the C ABI of
include/pthr.h); this package only binds it.
"""
from . import _lib  # noqa: F401
from .batch import Batch, BatchConfig, Group, required_bytes, buffer_info  # noqa: F401

__all__ = ["Batch", "BatchConfig", "Group", "required_bytes", "buffer_info"]
