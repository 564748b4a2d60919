"""GB300 (sm_103a) structured sparse QR for the damped least-squares step of LM.

The numerical work lives in the C-ABI library libqrkit.so (include/qrkit.h); this package
holds the CUDA sources (csrc/), the in-tree build (build.py) and the ctypes binding
(qrkit.py).
"""
from . import qrkit  # noqa: F401
from .qrkit import Context, QRKitError, load  # noqa: F401
