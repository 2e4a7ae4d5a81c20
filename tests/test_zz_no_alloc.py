"""qpr_rhs_noalloc against qpr_rhs.

qpr_rhs_noalloc serves callers that cannot allocate device memory (hosts
that own every device allocation through their own pool, fixed memory
budgets, no allocation after start-up): it keeps its scratch in a
fixed-size __device__ array and takes everything else from the caller. This
test builds the CSR operands from the CPU oracle's operators, calls the
entry point through the C ABI for three sizes in a row, twice each (every
call runs on the scratch the previous one left behind, a larger size's
included), and checks every output against the context-based qpr_rhs and
the oracle's right-hand side within the tolerance of the other
right-hand-side parity tests. The file name sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _csr(M):
    rows, cols = np.nonzero(M)
    ptr = np.zeros(M.shape[0] + 1, dtype=np.int32)
    np.add.at(ptr, rows + 1, 1)
    return np.cumsum(ptr).astype(np.int32), cols.astype(np.int32), M[rows, cols].astype(np.float64)


def _operands(g, **kw):
    """CSR of H and of S (columns with out-links) plus the dangling flags,
    from the oracle's adjacency and Hamiltonian, on the device."""
    o = Oracle.from_edges(g, **kw)
    A, H, G, c = o.operators()
    outdeg = A.sum(axis=0)
    S = np.zeros_like(A)
    has = outdeg > 0
    S[:, has] = A[:, has] / outdeg[has]
    hp, hc, hv = _csr(H)
    sp, sc, sv = _csr(S)
    dang = (~has).astype(np.uint8)
    return [torch.from_numpy(x).to(DEV) for x in (hp, hc, hv, sp, sc, sv, dang)]


def _call(lib, n, ops, alpha, omega, dangling, rho, out):
    p = [ctypes.c_void_p(t.data_ptr()) for t in ops]
    return lib.qpr_rhs_noalloc(n, p[0], p[1], p[2], p[3], p[4], p[5], p[6], alpha, omega, dangling,
                               ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


CASES = [(256, 0.0, 0), (97, 0.3, 1), (200, 0.8, 0)]


def _graph(n):
    return graphs.heavy_tailed(n, 11) if n != 97 else graphs.erdos_renyi(n, 0.03, 5)


def test_noalloc_rhs_matches_context_rhs_twice():
    # one test, sizes in the order 256, 97, 200: each call runs on the scratch
    # the previous one left behind, including a larger padded size's (256 ->
    # 128 -> 224 padded rows), and each size is called twice in a row
    lib = Q.load_library()
    for n, omega, dangling in CASES:
        g = _graph(n)
        kw = dict(alpha=0.85, omega=omega, dangling=dangling)
        ops = _operands(g, **kw)
        s = Solver.from_edges(g, **kw)
        o = Oracle.from_edges(g, **kw)
        for call in range(2):
            rho = torch.from_numpy(graphs.random_hermitian(n, 100 + call)).to(DEV)
            ref = torch.zeros_like(rho)
            s.rhs(rho, ref)
            out = torch.full_like(rho, float("nan"))
            assert _call(lib, n, ops, 0.85, omega, dangling, rho, out) == Q.QPR_OK
            torch.cuda.synchronize()
            r, got = ref.cpu().numpy(), out.cpu().numpy()
            scale = max(1.0, np.abs(r).max())
            assert np.abs(got - r).max() <= 1e-13 * scale * max(1, n / 16), (n, call)
            # and directly against the oracle's right-hand side
            f = o.rhs(rho.cpu().numpy())
            assert np.abs(got - f).max() <= 1e-13 * max(1.0, np.abs(f).max()) * max(1, n / 16), (n, call)
        s.close()


def test_noalloc_rejects_sizes_beyond_maximum():
    lib = Q.load_library()
    n = Q.QPR_NOALLOC_MAX_N + 1
    dummy = torch.zeros(4, dtype=torch.float64, device=DEV)
    ops = [dummy] * 7
    rho = torch.zeros((n, n), dtype=torch.complex128, device=DEV)
    assert _call(lib, n, ops, 0.85, 0.5, 0, rho, rho.clone()) == Q.QPR_E_ARG
    assert _call(lib, 1, ops, 0.85, 0.5, 0, rho, rho.clone()) == Q.QPR_E_ARG
