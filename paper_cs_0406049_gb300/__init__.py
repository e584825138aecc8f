"""GB300-native (sm_103a) branch-free single-precision sine-cosine pairs.

The method is M. H. Mendenhall's (cs/0406049): scale by 1/(2 pi), reduce by
rounding and subtraction, quarter-angle power series, two double-angle steps
of Eq. (1) and an amplitude-drift correction.  It runs in hand-written CUDA
kernels behind the C ABI of ``include/sincos_pairs.h``; this package is the
thin Python binding (``api``), the in-tree build (``build``) and the seeded
input generators (``workloads``).  Importing it does not load the CUDA
library; the first call does, and fails loudly if it is missing.
"""
__all__ = ["api", "build", "workloads"]
