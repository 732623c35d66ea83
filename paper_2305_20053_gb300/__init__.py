"""GB300-native (sm_103a) SAA risk + gradient engine for PDE-constrained
optimisation under uncertainty (arXiv 2305.20053).

The compute lives in libouu.so (CUDA kernels behind the C ABI of include/ouu.h);
`capi` is the thin ctypes binding with the same call names.
"""
from . import capi  # noqa: F401

__all__ = ["capi"]
