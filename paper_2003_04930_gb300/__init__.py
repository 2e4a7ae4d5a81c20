"""GB300 (sm_103a) solver for quantum PageRank.

Classical RK4 on the quantum-stochastic-walk Lindblad equation (Eq. 1 /
Eq. S7 of "TensorFlow Solver for Quantum PageRank in Large-Scale Networks"),
run directly on the N x N density matrix by hand-written CUDA kernels behind
the C ABI of ``include/qpr.h``.

  * ``qpr``    -- the ctypes binding (``Solver``) of ``_build/libqpr.so``
  * ``graphs`` -- seeded synthetic graph / initial-state generators
  * ``build``  -- nvcc build of the library
"""
from . import graphs  # noqa: F401
from .qpr import QprError, Solver, load_library  # noqa: F401
