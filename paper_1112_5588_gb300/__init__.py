"""GB300-native pJDS sparse matrix-vector multiplication.

y = A x with A in padded jagged diagonals storage (pJDS) and in ELLPACK-R, after
Kreutzer et al., "Sparse matrix-vector multiplication on GPGPU clusters: A new
storage format and a scalable implementation" (arXiv:1112.5588).

Modules:
  pjds       ctypes binding of libpjds.so (the C ABI in include/pjds.h)
  perfmodel  the paper's code-balance and PCIe-transfer model (Eqs. 1-4)
  build      compiles libpjds.so for sm_103a
"""
__version__ = "0.1.0"
