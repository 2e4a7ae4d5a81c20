"""GPU parity of the dense mixed form: split-BF16 tcgen05 stage GEMM.

The 3-term BF16 split represents H and the FP32 stage delta to about 2^-24
and the six products accumulate in FP32, so the stage deltas carry FP32-level
error, exactly like the sparse FP32 kernel of the mixed form, and the steady
state is polished by exact FP64 refreshes. Away from equilibrium the error
per unit time is about eps ||L|| (ref_refresh dt) ||f|| (derivation in
tests/test_gpu_mixed.py), and the 40-step trajectories are held to
||drho||_F <= 1e-6. The tensor core's FP32 accumulation does not round to
nearest, so its error grows with the K-steps added to a large accumulator;
with the small split products accumulated before the dominant H0 d0 product
the measured error is 1.5-5x that of the FP32 sparse kernel on the same
trajectory (25-70x with H0 d0 first), and the test requires at most 8x. Sizes cover a single diagonal
128-tile (N = 100), the unpadded multiple (N = 256) and several tile pairs
with a ragged tail (N = 300).
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle.cpu import populations
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _dense_graph(n, seed, p=0.15):
    g = graphs.erdos_renyi(n, p, seed)
    w = np.random.default_rng(seed + 7).lognormal(0.0, 1.0, g.m)
    return graphs.EdgeList(g.n, g.src, g.dst, w)


def _tc(g, **kw):
    s = Solver.from_edges(g, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_DENSE, **kw)
    assert s.backend == Q.QPR_BACKEND_DENSE
    return s


@pytest.mark.parametrize("n", [100, 256, 300])
@pytest.mark.parametrize("omega", [0.3, 0.8])
def test_tc_trajectory_parity(n, omega):
    g = _dense_graph(n, 3)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    s = _tc(g, alpha=0.85, omega=omega, ref_refresh=2)
    sp = Solver.from_edges(g, alpha=0.85, omega=omega, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                           ref_refresh=2)
    rho0 = graphs.random_density(n, 4, rank=3)
    dt = min(0.01, 0.5 * s.max_stable_dt)
    ref = o.evolve(rho0, dt, 40)
    d = _dev(rho0)
    s.evolve(d, dt, 40)
    got = d.cpu().numpy()
    d2 = _dev(rho0)
    sp.evolve(d2, dt, 40)
    err_tc = np.linalg.norm(got - ref)
    err_sp = np.linalg.norm(d2.cpu().numpy() - ref)
    p, pr = populations(got), populations(ref)
    assert err_tc <= 1e-6, (err_tc, err_sp)
    assert err_tc <= 8.0 * err_sp + 1e-9, (err_tc, err_sp)
    assert np.abs(p - pr).max() <= 1e-6 * pr.max()
    assert np.abs(got - got.conj().T).max() == 0.0


def test_tc_heavy_tailed_matches_sparse_mixed():
    g = graphs.heavy_tailed(300, 1)
    rho0 = graphs.random_density(300, 9, rank=2)
    outs = []
    for be in (Q.QPR_BACKEND_DENSE, Q.QPR_BACKEND_SPARSE):
        s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, backend=be, ref_refresh=16)
        d = _dev(rho0)
        s.evolve(d, 0.01, 64)
        outs.append(d.cpu().numpy())
    ref = Oracle.from_edges(g, alpha=0.85, omega=0.8).evolve(rho0, 0.01, 64)
    for got in outs:
        assert np.linalg.norm(got - ref) <= 1e-6
    assert np.linalg.norm(outs[0] - outs[1]) <= 1e-6


def test_tc_steady_state():
    g = _dense_graph(200, 5, p=0.2)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    s = _tc(g, alpha=0.85, omega=0.8)
    dt = min(0.01, 0.5 * s.max_stable_dt)
    rho0 = graphs.maximally_mixed(200)
    ref, steps_ref, r_ref, st = o.steady_state(rho0, dt, 1e-8, 200000)
    assert st == 0
    d = _dev(rho0)
    stats = s.steady_state(d, dt, 1e-8, 200000)
    assert stats["converged"] == 1 and stats["residual"] < 1e-8
    assert abs(stats["steps"] - steps_ref) <= 1
    got = d.cpu().numpy()
    p, pr = populations(got), populations(ref)
    assert np.linalg.norm(got - ref) <= 1e-6
    assert np.abs(p - pr).max() <= 1e-7 * pr.max()
