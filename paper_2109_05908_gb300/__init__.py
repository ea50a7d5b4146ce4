"""GB300 (sm_103a) implementation of the two-level algebraic overlapping
Schwarz preconditioner of Al Daas & Jolivet (arXiv 2109.05908).

The numerical work lives in the CUDA library libamdd.so (C ABI in
include/amdd.h); `amdd` is its thin ctypes binding and `device` moves seeded
host inputs into CUDA memory owned by torch.
"""
