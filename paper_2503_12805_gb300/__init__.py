"""GB300 (sm_103a) implementation of the fast Fourier spectral evaluation of the
4-wave kinetic collision operator (Qi, Shen, Wang, arXiv 2503.12805).

The compute path is the C-ABI library ``libwke.so`` (CUDA kernels); ``wke``
is its Python binding.  ``build`` compiles the library in-tree.
"""
from .build import build  # noqa: F401
