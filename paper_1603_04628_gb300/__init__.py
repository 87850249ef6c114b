"""GB300-native micro-MD + Gaussian-process hybrid flow library (arXiv:1603.04628).

The compute path lives in libmdgp.so (CUDA, sm_103a); this package only
builds it and marshals arguments.  See include/mdgp.h for the C ABI."""
from . import native  # noqa: F401
from .native import Context, MdgpError, PREC_FP32, PREC_FP64  # noqa: F401
