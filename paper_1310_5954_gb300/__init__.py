"""GB300 (sm_103a) local ETKF control law for adaptive optics (arXiv:1310.5954).

The compute path is libletkf.so: hand-written CUDA kernels behind the C ABI of
include/letkf.h.  This package holds the ctypes binding (`_lib`, same names as
the C ABI), a thin class that marshals torch device tensors (`LETKF`), the
in-tree build (`build`), and the multi-system serving loop (`serve.Server`, over
include/letkf_serve.h).
PyTorch is used for device memory and streams only.
"""

from ._lib import (LETKF_PATH_FUSED, LETKF_PATH_PLAIN, LETKF_PREC_FP32, LETKF_PREC_FP64,  # noqa: F401
                   LETKF_PREC_MIXED, LETKFError, load)
from .letkf import LETKF, LETKFPair, footprint  # noqa: F401
from .serve import Server  # noqa: F401
