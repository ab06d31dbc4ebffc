"""GB300 (sm_103a) implementation of the structure-preserving H(curl) AMG method (SpHcurlAMG)
for the lowest-order edge-element eddy-current system, behind the C ABI of include/sphc.h.

``sphc`` is the ctypes binding of libsphc.so; ``build`` compiles it with nvcc.
"""
from . import build, sphc  # noqa: F401

__all__ = ["build", "sphc"]
