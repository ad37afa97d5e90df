"""GB300-native short-range molecular dynamics (cell/neighbour-list pair forces).

The compute path is the CUDA library ``libgbmd.so`` (hand-written kernels for sm_103a behind a
C ABI, declared in ``include/gbmd.h``).  ``binding`` loads it and exposes the same entry points;
``system`` wraps them with torch-owned device memory.  Nothing in this package falls back to a
CPU implementation: if the library is missing, loading fails with an error.
"""
__all__ = ["inputs"]
