"""GB300-native wavelet-Sobolev / Matern photoacoustic reconstruction.

The compute path is libpat.so (hand-written sm_103a CUDA behind the C ABI of
include/pat.h).  This package is the thin Python side: the ctypes binding
(`_lib`, same names as the C ABI), a `Plan` convenience wrapper and the
torch.autograd wrappers (`autograd`).  PyTorch supplies device memory and
streams only.
"""
from . import _lib  # noqa: F401
from ._lib import PatError, PAT_PATH_AUTO, PAT_PATH_PERSISTENT, PAT_PATH_STEP  # noqa: F401
from .plan import Batch, Plan  # noqa: F401
