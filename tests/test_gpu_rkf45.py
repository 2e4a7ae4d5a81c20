"""qpr_rkf45 (adaptive RKF45, Supplementary Note 2) against the oracle's RKF45.

The oracle takes the six stages of Eq. S10 literally in FP64; the library
evaluates the same polynomial of h L from its powers in the mixed delta form
and runs the controller on the device. Both use the same h0, Tol and h_max.
The accept/reject decisions are comparisons of the discrepancy with Tol h;
the two sides compute the discrepancy in different precisions (FP64 against
FP32 powers), so a decision could differ only for a discrepancy within ~1e-6
relative of Tol h: the tests compare step counts within a small slack and the
states within the mixed form's bounds (trajectories ||drho||_F <= 1e-6 and
max|dp| <= 1e-6 max p; steady states max|dp| <= 1e-7 max p). The returned
residual is the exact FP64 one.
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


def _solver(g, omega, form=Q.QPR_SPARSE_FORM_AUTO, refresh=32):
    return Solver.from_edges(g, alpha=0.85, omega=omega, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                             sparse_form=form, ref_refresh=refresh)


def _close(got, ref, prel):
    p, pr = populations(got), populations(ref)
    assert np.linalg.norm(got - ref) <= 1e-6
    assert np.abs(p - pr).max() <= prel * pr.max()


@pytest.mark.parametrize("n,omega,form,refresh,order", [(33, 0.8, Q.QPR_SPARSE_FORM_COLUMNS, 32, 4),
                                                        (200, 0.3, Q.QPR_SPARSE_FORM_COLUMNS, 7, 4),
                                                        (200, 0.3, Q.QPR_SPARSE_FORM_COLUMNS, 7, 5),
                                                        (520, 0.6, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, 16, 5),
                                                        (300, 0.8, Q.QPR_SPARSE_FORM_COLUMNS_GATHER, 32, 4)])
def test_rkf45_trajectory_matches_oracle(n, omega, form, refresh, order):
    g = graphs.heavy_tailed(n, 5)
    s = _solver(g, omega, form, refresh)
    hmax = s.max_stable_dt
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.random_density(n, 4, rank=3)
    t_end = 1.5
    ref = o.rkf45(rho0, 0.01, 1e-6, hmax, t_end=t_end, max_steps=5000, order=order)
    d = torch.from_numpy(rho0.copy()).to(DEV)
    st = s.rkf45(d, h0=0.01, step_tol=1e-6, h_max=hmax, t_end=t_end, max_steps=5000, order=order)
    assert st["converged"] == 1 and st["t"] == pytest.approx(t_end, rel=1e-14)
    assert abs(st["accepted"] - ref["accepted"]) <= 2 and abs(st["rejected"] - ref["rejected"]) <= 2
    got = d.cpu().numpy()
    _close(got, ref["rho"], 1e-6)
    assert np.abs(got - got.conj().T).max() == 0.0
    assert abs(np.trace(got).real - 1.0) < 1e-13


def test_rkf45_rejections_follow_the_oracle():
    # a first step far too large for Tol: the controller rejects and shrinks h
    g = graphs.heavy_tailed(150, 3)
    s = _solver(g, 0.5)
    hmax = s.max_stable_dt
    o = Oracle.from_edges(g, alpha=0.85, omega=0.5)
    rho0 = graphs.random_density(150, 8, rank=1)
    ref = o.rkf45(rho0, hmax, 1e-9, hmax, t_end=0.5, max_steps=5000)
    assert ref["rejected"] >= 1
    d = torch.from_numpy(rho0.copy()).to(DEV)
    st = s.rkf45(d, h0=hmax, step_tol=1e-9, h_max=hmax, t_end=0.5, max_steps=5000)
    assert st["rejected"] >= 1 and abs(st["rejected"] - ref["rejected"]) <= 2
    assert abs(st["accepted"] - ref["accepted"]) <= 2
    _close(d.cpu().numpy(), ref["rho"], 1e-6)


# steady states: order 4 at omega = 0.8, order 5 (the note's alternative)
# also at omega = 0.5, where the fourth-order solution stalls (see qpr.h)
@pytest.mark.parametrize("n,omega,order", [(150, 0.8, 4), (150, 0.8, 5), (200, 0.5, 5)])
def test_rkf45_steady_state_matches_oracle(n, omega, order):
    g = graphs.heavy_tailed(n, 6)
    s = _solver(g, omega)
    hmax = s.max_stable_dt
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.maximally_mixed(n)
    ref = o.rkf45(rho0, 0.01, 1e-6, hmax, resid_tol=1e-8, max_steps=20000, order=order)
    assert ref["status"] == 0
    d = torch.from_numpy(rho0.copy()).to(DEV)
    st = s.rkf45(d, tol=1e-8, h0=0.01, step_tol=1e-6, h_max=hmax, max_steps=20000, order=order)
    got = d.cpu().numpy()
    assert st["converged"] == 1 and st["residual"] < 1e-8
    assert abs(st["residual"] - o.residual(got)) <= 1e-12
    assert abs(st["accepted"] - ref["accepted"]) <= 2
    _close(got, ref["rho"], 1e-7)
    # fewer steps than fixed-step RK4 at dt = 0.01 to the same tolerance, same steady state
    _, rk4_steps, _, _ = o.steady_state(rho0, 0.01, 1e-8, 200000)
    assert st["accepted"] < rk4_steps


def test_rkf45_steady_state_equals_rk4_steady_state_polished():
    g = graphs.heavy_tailed(250, 9)
    s = _solver(g, 0.7)
    d = torch.from_numpy(graphs.maximally_mixed(250)).to(DEV)
    s.rkf45(d, tol=1e-11, max_steps=20000, order=5)
    r = torch.from_numpy(graphs.maximally_mixed(250)).to(DEV)
    s.steady_state(r, 0.01, 1e-11, 200000)
    a, b = d.cpu().numpy(), r.cpu().numpy()
    assert np.abs(populations(a) - populations(b)).max() <= 1e-7 * populations(b).max()
    assert np.linalg.norm(a - b) <= 1e-6


def test_rkf45_max_steps_and_arguments():
    g = graphs.heavy_tailed(100, 2)
    s = _solver(g, 0.8)
    d = torch.from_numpy(graphs.maximally_mixed(100)).to(DEV)
    st = s.rkf45(d, tol=1e-13, max_steps=5, check=False)
    assert st["status"] == Q.QPR_E_NOT_CONVERGED and st["accepted"] == 5
    fp64 = Solver.from_edges(g, alpha=0.85, omega=0.8)
    with pytest.raises(Q.QprError) as e:
        fp64.rkf45(d, tol=1e-8)
    assert e.value.status == Q.QPR_E_ARG
    tiles = _solver(g, 0.8, Q.QPR_SPARSE_FORM_TILES)
    with pytest.raises(Q.QprError) as e:
        tiles.rkf45(d, tol=1e-8)
    assert e.value.status == Q.QPR_E_ARG
    with pytest.raises(Q.QprError) as e:
        s.rkf45(d, tol=0.0)
    assert e.value.status == Q.QPR_E_ARG
    with pytest.raises(Q.QprError) as e:
        s.rkf45(d, tol=1e-8, order=3)
    assert e.value.status == Q.QPR_E_ARG
