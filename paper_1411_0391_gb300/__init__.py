"""GB300 (sm_103a) implementation of iPEPS imaginary-time evolution with CTMRG
environments, full-update truncation and environment recycling
(Phien, McCulloch, Vidal, arXiv:1411.0391).

The compute path is libtnite.so (CUDA, C ABI in include/tnite.h); the Python
side only marshals arguments (_lib) and builds the library (build).  Importing
this package loads nothing; the library is loaded on first use.
"""
__all__ = ["build", "inputs"]
