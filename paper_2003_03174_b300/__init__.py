"""B300-native (sm_103a) TRD tracklet follower (arXiv:2003.03174, Sec. 3).

The compute path is libtrd.so: hand-written FP32 CUDA kernels behind the C
ABI of include/trd_abi.h.  `trd` is the thin Python binding over it.
"""
from . import trd  # noqa: F401

__all__ = ["trd"]
