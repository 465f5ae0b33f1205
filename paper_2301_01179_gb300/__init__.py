"""GB300-native (sm_103a) cylindrical-coordinate FMM for modal ring sources.

Carley, "A Fast Multipole Method for axisymmetric domains" (arXiv 2301.01179): the
Fourier modes n = 0..N of the potential of azimuthally varying ring sources, evaluated
at field points (r, z) directly and by a uniform quadtree FMM.

The compute path is the C-ABI library ``libafmm.so`` (CUDA kernels for sm_103a, header
``include/afmm.h``); :mod:`.binding` marshals torch device tensors into it and
:mod:`.autograd` wraps forward and adjoint in a ``torch.autograd.Function``.  Importing
this package does not load the library; the first call does, and fails loudly if the
library has not been built.
"""
__all__ = ["binding", "workloads"]
