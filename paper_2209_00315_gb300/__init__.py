"""GB300 solver for Benamou-Brenier dynamical optimal transport by interior points.

The path (Facca, Todeschi, Natale, Benzi, arXiv 2209.00315): an interior-point
method whose Newton systems are solved by flexible GMRES preconditioned with
the BB approximation of the Schur complement, all in hand-written CUDA kernels
behind the C ABI of ``include/ot.h``.  ``capi`` is the ctypes binding with the
same function names; ``autograd`` wraps the solve and the adjoint gradient in
a ``torch.autograd.Function``.
"""
from . import capi  # noqa: F401

__all__ = ["capi"]
