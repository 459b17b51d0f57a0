"""GB300-native (sm_103a) plain-LRSTV hyperspectral denoiser (arXiv 2204.12879).

The computation lives in ``liblrstv.so`` (hand-written CUDA behind the C ABI
of ``include/lrstv.h``); this package builds it in-tree and binds it with
ctypes.  There is no CPU path.
"""
from .builder import build  # noqa: F401
from .lrstv import *  # noqa: F401,F403
from .lrstv import __all__ as _all

__all__ = ["build", *_all]
