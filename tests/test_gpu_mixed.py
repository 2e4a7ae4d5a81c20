"""GPU parity of the mixed-precision form (QPR_MIXED) against the FP64 oracle.

Steady states are held to the precision form's bounds: ||rho_gpu - rho||_F
<= 1e-6 and max_i |p_gpu,i - p_i| <= 1e-7 max_i p_i (residual 1e-8, the
returned state re-checked by an exact FP64 residual).

Trajectories far from equilibrium carry the FP32 error of the stage deltas:
per unit time about eps32 * ||L|| * (ref_refresh * dt) * ||f||, with
eps32 = 6e-8, ||L|| the generator's norm (about the spread of H, ~1e2 here),
ref_refresh * dt <= 0.32 and ||f|| <= 0.1 away from equilibrium: at most
~2e-7 per unit time, i.e. ~3e-7 over the 150-step (t = 1.5) trajectories and
~2e-5 over t = 100. They are held to ||drho||_F <= 1e-6 and
max|dp| <= 1e-6 max p (t = 1.5), and to the 1e-7 bound once the state has
relaxed (the 10^4-step config-1 trajectory ends at equilibrium).
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle.cpu import populations
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_steady_n922.json")


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _mixed(g, **kw):
    return Solver.from_edges(g, precision=Q.QPR_MIXED, **kw)


def _close(got, ref, prel=1e-7):
    p, pr = populations(got), populations(ref)
    assert np.linalg.norm(got - ref) <= 1e-6
    assert np.abs(p - pr).max() <= prel * pr.max()


@pytest.mark.parametrize("n", [16, 97, 200])
@pytest.mark.parametrize("omega", [0.2, 0.8, 1.0])
@pytest.mark.parametrize("refresh", [1, 7, 32])
def test_mixed_trajectory_parity(n, omega, refresh):
    g = graphs.heavy_tailed(n, 1) if n > 16 else graphs.erdos_renyi(16, 0.25, 0)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    s = _mixed(g, alpha=0.85, omega=omega, ref_refresh=refresh)
    rho0 = graphs.random_density(n, 3, rank=2)
    ref = o.evolve(rho0, 0.01, 150)
    d = _dev(rho0)
    s.evolve(d, 0.01, 150)
    got = d.cpu().numpy()
    _close(got, ref, prel=1e-6)
    assert np.abs(got - got.conj().T).max() == 0.0
    assert abs(np.trace(got).real - 1.0) < 1e-14


def test_mixed_config1_full_trajectory():
    g = graphs.erdos_renyi(16, 0.25, 0)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    s = _mixed(g, alpha=0.85, omega=0.8)
    rho0 = graphs.maximally_mixed(16)
    ref = o.evolve(rho0, 0.01, 10000)
    d = _dev(rho0)
    s.evolve(d, 0.01, 10000)
    _close(d.cpu().numpy(), ref)


@pytest.mark.parametrize("n,omega", [(48, 0.8), (150, 0.5), (150, 1.0)])
def test_mixed_steady_state(n, omega):
    g = graphs.heavy_tailed(n, 2)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.maximally_mixed(n)
    ref, steps_ref, r_ref, st = o.steady_state(rho0, 0.01, 1e-8, 200000)
    assert st == 0
    s = _mixed(g, alpha=0.85, omega=omega)
    d = _dev(rho0)
    stats = s.steady_state(d, 0.01, 1e-8, 200000)
    assert stats["converged"] == 1 and stats["residual"] < 1e-8
    assert abs(stats["steps"] - steps_ref) <= 1
    got = d.cpu().numpy()
    _close(got, ref)
    # the reported residual is the exact FP64 residual of the returned state
    assert abs(stats["residual"] - o.residual(got)) <= 1e-12


@pytest.mark.parametrize("n,omega", [(150, 0.5), (400, 0.8)])
def test_adaptive_refresh_window(n, omega):
    # steady states with the lengthening refresh window (default) and with a
    # refresh every ref_refresh steps: both within the precision form's
    # bounds of the oracle, the same step count within 1, fewer launches
    g = graphs.heavy_tailed(n, 3)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.maximally_mixed(n)
    ref, steps_ref, _, _ = o.steady_state(rho0, 0.01, 1e-8, 200000)
    got, stats = {}, {}
    for adaptive in (0, 1):
        s = _mixed(g, alpha=0.85, omega=omega, backend=Q.QPR_BACKEND_SPARSE, adaptive_refresh=adaptive)
        d = _dev(rho0)
        stats[adaptive] = s.steady_state(d, 0.01, 1e-8, 200000)
        got[adaptive] = d.cpu().numpy()
        assert stats[adaptive]["converged"] == 1 and stats[adaptive]["residual"] < 1e-8
        assert abs(stats[adaptive]["steps"] - steps_ref) <= 1
        assert abs(stats[adaptive]["residual"] - o.residual(got[adaptive])) <= 1e-12
        _close(got[adaptive], ref)
    assert stats[1]["kernel_launches"] < stats[0]["kernel_launches"]


def test_mixed_not_converged_and_zero_steps():
    g = graphs.heavy_tailed(60, 5)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.5)
    s = _mixed(g, alpha=0.85, omega=0.5, ref_refresh=8)
    rho0 = graphs.random_density(60, 1)
    d = _dev(rho0)
    stats = s.steady_state(d, 0.01, 1e-12, 37, check=False)
    assert stats["status"] == Q.QPR_E_NOT_CONVERGED and stats["steps"] == 37
    ref = o.evolve(rho0, 0.01, 37)
    got = d.cpu().numpy()
    _close(got, ref, prel=1e-6)
    # the reported residual is the exact FP64 residual of the returned state
    assert abs(stats["residual"] - o.residual(got)) <= 1e-12 * max(1.0, stats["residual"])
    d0 = _dev(rho0)
    s.evolve(d0, 0.01, 0)
    np.testing.assert_allclose(d0.cpu().numpy(), rho0 / np.trace(rho0).real, rtol=0, atol=1e-16)


def test_mixed_nan_reported():
    g = graphs.heavy_tailed(40, 1)
    s = _mixed(g, alpha=0.85, omega=0.5)
    x = graphs.maximally_mixed(40)
    x[2, 7] = np.nan
    stats = s.steady_state(_dev(x), 0.01, 1e-8, 50, check=False)
    assert stats["status"] == Q.QPR_E_NONFINITE


@pytest.mark.parametrize("precision", [Q.QPR_FP64, Q.QPR_MIXED])
@pytest.mark.parametrize("omega", [0.8, 1.0])
def test_airline_size_steady_state_against_stored_oracle(precision, omega):
    # N = 922, seed 1, rho0 = I/N, dt = 0.01, tol 1e-8: the oracle's step
    # count and populations were written by tests/golden/make_oracle_steady_states.py
    gold = json.load(open(GOLDEN))[str(omega)]
    g = graphs.heavy_tailed(922, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=omega, precision=precision)
    d = _dev(graphs.maximally_mixed(922))
    stats = s.steady_state(d, 0.01, 1e-8, 400000)
    assert stats["converged"] == 1
    assert abs(stats["steps"] - gold["steps"]) <= 1
    p = populations(d.cpu().numpy())
    pr = np.array(gold["populations"])
    assert np.abs(p - pr).max() <= 1e-7 * pr.max()


def test_mixed_matches_fp64_form_bitwise_independent_of_graphs():
    g = graphs.heavy_tailed(80, 4)
    rho0 = _dev(graphs.random_density(80, 5))
    outs = []
    for gs in (0, 32):
        s = Solver.from_edges(g, alpha=0.85, omega=0.5, precision=Q.QPR_MIXED, graph_steps=gs, ref_refresh=16)
        r = rho0.clone()
        st = s.steady_state(r, 0.01, 1e-6, 100000)
        outs.append((st["steps"], r.cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
