"""Parity at the second benchmark size, N = 4096 (heavy-tailed graph, seed 3,
omega = 0.8), in the launch configuration bench.py times: the mixed form with
the default plan (gather SpMM, 14 row splits, cut hub rows), captured CUDA
graphs and programmatic dependent launch.

  * a 24-step RK4 trajectory from a random rank-3 density matrix against the
    FP64 oracle (||drho||_F <= 1e-6, max|dp| <= 1e-6 max p; it crosses an
    exact FP64 refresh);
  * single right-hand-side entries f(rho)_ij at sampled (i, j), from the
    oracle's f on the same state (qpr_rhs through the FP64 form of the same
    graph, at 1e-12 of max |f|);
  * the properties every state keeps at any size: unit trace, exact
    Hermiticity, and for the steady state the exact FP64 residual below the
    tolerance, with the populations of the FP64 sparse form's steady state;
  * a short RKF45 trajectory (fifth order, to t = 0.25) against the oracle's
    RKF45, accepted and rejected attempts within 2.
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
N, SEED, OMEGA = 4096, 3, 0.8


@pytest.fixture(scope="module")
def graph():
    return graphs.heavy_tailed(N, SEED)


def test_trajectory_at_n4096_against_oracle(graph):
    rho0 = graphs.random_density(N, 7, rank=3)
    steps = 24
    ref = Oracle.from_edges(graph, alpha=0.85, omega=OMEGA).evolve(rho0, 0.01, steps)
    s = Solver.from_edges(graph, alpha=0.85, omega=OMEGA, precision=Q.QPR_MIXED, ref_refresh=16)
    assert s.sparse_form == Q.QPR_SPARSE_FORM_COLUMNS_GATHER
    d = torch.from_numpy(rho0.copy()).to(DEV)
    s.evolve(d, 0.01, steps)
    got = d.cpu().numpy()
    p, pr = populations(got), populations(ref)
    assert np.linalg.norm(got - ref) <= 1e-6
    assert np.abs(p - pr).max() <= 1e-6 * pr.max()
    assert np.abs(got - got.conj().T).max() == 0.0
    assert abs(np.trace(got).real - 1.0) < 1e-13


def test_rhs_entries_at_n4096_against_oracle(graph):
    rho = graphs.random_density(N, 11, rank=2)
    ref = Oracle.from_edges(graph, alpha=0.85, omega=OMEGA).rhs(rho)
    s = Solver.from_edges(graph, alpha=0.85, omega=OMEGA)  # the FP64 sparse form
    x = torch.from_numpy(rho).to(DEV)
    out = torch.empty_like(x)
    got = s.rhs(x, out).cpu().numpy()
    rng = np.random.default_rng(5)
    ii, jj = rng.integers(0, N, 4000), rng.integers(0, N, 4000)
    scale = np.abs(ref).max()
    assert np.abs(got[ii, jj] - ref[ii, jj]).max() <= 1e-12 * scale
    assert np.abs(np.diag(got) - np.diag(ref)).max() <= 1e-12 * scale


def test_steady_state_properties_at_n4096(graph):
    s = Solver.from_edges(graph, alpha=0.85, omega=OMEGA, precision=Q.QPR_MIXED)
    d = torch.from_numpy(graphs.maximally_mixed(N)).to(DEV)
    st = s.steady_state(d, 0.01, 1e-8, 100000)
    assert st["converged"] == 1 and st["residual"] < 1e-8
    got = d.cpu().numpy()
    assert np.abs(got - got.conj().T).max() == 0.0
    assert abs(np.trace(got).real - 1.0) < 1e-13
    f64 = Solver.from_edges(graph, alpha=0.85, omega=OMEGA)
    r = torch.from_numpy(graphs.maximally_mixed(N)).to(DEV)
    st64 = f64.steady_state(r, 0.01, 1e-8, 100000)
    assert abs(st64["steps"] - st["steps"]) <= 1
    p, p64 = populations(got), populations(r.cpu().numpy())
    assert np.abs(p - p64).max() <= 1e-7 * p64.max()


def test_rkf45_trajectory_at_n4096_against_oracle(graph):
    # the paper's integrator in the same plan (gather SpMM): a short adaptive
    # trajectory to t = 0.25 against the oracle's RKF45 (same h0, Tol, h_max)
    s = Solver.from_edges(graph, alpha=0.85, omega=OMEGA, precision=Q.QPR_MIXED)
    hmax = s.max_stable_dt
    rho0 = graphs.random_density(N, 13, rank=2)
    ref = Oracle.from_edges(graph, alpha=0.85, omega=OMEGA).rkf45(rho0, 0.01, 1e-6, hmax, t_end=0.25,
                                                                   max_steps=200, order=5)
    d = torch.from_numpy(rho0.copy()).to(DEV)
    st = s.rkf45(d, h0=0.01, step_tol=1e-6, h_max=hmax, t_end=0.25, max_steps=200, order=5)
    assert st["converged"] == 1 and st["t"] == pytest.approx(0.25, rel=1e-14)
    assert abs(st["accepted"] - ref["accepted"]) <= 2 and abs(st["rejected"] - ref["rejected"]) <= 2
    got = d.cpu().numpy()
    p, pr = populations(got), populations(ref["rho"])
    assert np.linalg.norm(got - ref["rho"]) <= 1e-6
    assert np.abs(p - pr).max() <= 1e-6 * pr.max()
    assert np.abs(got - got.conj().T).max() == 0.0
