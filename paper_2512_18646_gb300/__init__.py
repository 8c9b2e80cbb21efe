"""GB300 (sm_103a) RNS-CKKS engine for the multi-ciphertext encrypted matrix
multiplication and convolution of "Volley Revolver ... (Inference++)"
(arXiv 2512.18646).

The compute path is the CUDA library libhegb300.so behind the C ABI in
include/he_gb300.h; `api` is a thin ctypes binding with the same names.
"""
from ._lib import HeError, load  # noqa: F401
from . import api  # noqa: F401
