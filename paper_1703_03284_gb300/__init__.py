"""GB300 (sm_103a) engine for the MIPWA Dalitz-plot likelihood of arXiv:1703.03284.

``Likelihood`` wraps the C ABI of libmipwa.so (include/mipwa.h); ``MipwaNLL`` is
its torch.autograd.Function; ``fit`` is the host quasi-Newton minimiser.
"""
from ._lib import F32, F64
from .api import Likelihood, MipwaError

__all__ = ["Likelihood", "MipwaError", "F32", "F64"]
