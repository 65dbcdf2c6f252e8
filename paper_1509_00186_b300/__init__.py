"""B300-native per-channel overlap-save coherent dedispersion (De & Gupta,
arXiv:1509.00186): a CUDA library with a C ABI (include/cdd.h) and a thin
Python binding (``cdd``)."""
__all__ = ["cdd", "build"]
