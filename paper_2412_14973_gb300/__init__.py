"""GB300 (sm_103a) library for reciprocity-aware tile low-rank MDD (arXiv 2412.14973).

The compute path is the C-ABI library ``lib/libtlr_mdd.so`` (hand-written CUDA);
``tlr_mdd`` is its ctypes binding and does argument marshalling only.  PyTorch
provides device memory and streams.  There is no CPU fallback: every call
fails loudly if the library is not built.
"""
from .tlr_mdd import *  # noqa: F401,F403
