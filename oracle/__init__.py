"""CPU oracle for the quantum PageRank RK4 path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The GPU library never imports, links
or calls anything here, and nothing here imports the GPU library.

Two parts:
  * ``cpu``     -- ctypes wrapper of ``qpr_oracle.c``: plain FP64 operator
                   assembly, the Lindblad right-hand side, classical RK4 and
                   the steady-state loop (OpenMP over rows, nothing else).
  * ``gnn``     -- FP64 forward/backward of the warm-start network.
  * ``superop`` -- NumPy construction of the N^2 x N^2 superoperator from the
                   N^2 jump operators (Eq. 2 / Eq. S8, Eq. 3 / Eq. S9) and its
                   exact solutions by eigendecomposition, for N <= 24.
"""
from .cpu import Oracle, OracleError, build_oracle_lib, oracle_lib_path  # noqa: F401
from . import gnn, superop  # noqa: F401
