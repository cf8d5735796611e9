"""GB300-native factorized quark propagator (Ce, Giusti, Schaefer, arXiv:1612.06424).

The CUDA library (csrc/, C ABI in include/lqcd.h) holds every step of the
path; ``lqcd`` is its ctypes binding and ``inputs`` the seeded synthetic
input generators.
"""
__all__ = ["lqcd", "inputs", "build"]
