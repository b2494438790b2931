"""GB300-native SPH hydro right-hand side (FleCSPH, arXiv 2007.03097).

The compute path lives in the CUDA library ``lib/libsph.so`` built from
``csrc/``; ``binding`` is a thin ctypes layer over its C ABI (declared in
``include/sph.h``).  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["binding", "inputs"]
