"""GB300-native MFA-DVR: direct volume rendering of MFA models.

The product is ``lib/libmfadvr.so`` (C ABI in ``include/mfadvr.h``) with its
CUDA kernels for sm_103a; ``mfadvr`` is its Python binding and ``workloads``
makes seeded synthetic inputs.  Nothing is loaded at import time.
"""
__all__ = ["mfadvr", "workloads", "build"]
