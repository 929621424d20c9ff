"""GB300-native GWAS sequence of generalized least-squares problems.

b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y for i = 1..m with X_i = (X_L | x_Ri)
(Fabregat-Traver, Aulchenko, Bientinesi, Eq. 1), computed by hand-written CUDA
kernels for sm_103a behind the C ABI declared in include/gls_gb300.h.

Importing the package loads nothing native; ``paper_1210_7325_gb300.gls``
loads the shared library on first use and raises if it is missing.
"""

__all__ = ["gls", "synth"]
