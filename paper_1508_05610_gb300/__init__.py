"""GB300-native leapfrog lattice-field hot path (LATfield2, arXiv:1508.05610).

The compute path is the CUDA library ``liblf2.so`` (C ABI in ``include/lf2.h``); ``lf2`` is its
thin ctypes binding and ``inputs`` the seeded synthetic input generators.
"""
__all__ = ["lf2", "inputs"]
