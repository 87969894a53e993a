"""GB300-native library of the L2-norm regularized WENO-IS Euler solver
(Zhu & Hu, arXiv 1908.02464).

The computation runs in hand-written CUDA kernels behind a C ABI
(``include/weno_is.h``); ``paper_1908_02464_gb300.weno`` is the thin ctypes
binding with the same entry-point names, and ``problems`` holds the seeded
initial data of the test problems.
"""
__all__ = ["problems", "weno"]
