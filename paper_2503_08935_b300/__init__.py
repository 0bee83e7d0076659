"""B300-native preconditioned Bi-CGSTAB Poisson solver (arxiv 2503.08935).

The solver lives in the CUDA library ``libpsolve.so`` (C ABI in
``include/psolve.h``); ``binding`` is its thin ctypes binding and ``inputs``
holds the seeded synthetic input generators.  Importing the package loads
nothing; the library is loaded on first use and its absence is an error.
"""
__all__ = ["binding", "inputs"]
