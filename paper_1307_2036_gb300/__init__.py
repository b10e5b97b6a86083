"""GB300-native tensor-product multigrid and line-preconditioned CG for the
elliptic model equation of Mueller & Scheichl (arXiv:1307.2036).

The solver lives in the CUDA library libellsolve.so behind the C ABI declared in
include/ellsolve.h; `paper_1307_2036_gb300.ellsolve` is its thin ctypes binding
(importing it fails loudly when the library has not been built).
"""
__all__ = ["ellsolve", "inputs"]
