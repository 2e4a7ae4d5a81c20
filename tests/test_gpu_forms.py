"""The forms of the FP32 sparse stage of QPR_MIXED: the column-block form
(two launches per stage), its persistent form (one cooperative launch per
block of steps), its gather form (rows of the block read from L2, for any
N) and the tile-pair form.

The two whole-block column forms run the same device arithmetic (row
products in entry order, the same gain and epilogue sums, the same stop
decision), so their states, step counts and residuals are bitwise equal.
The gather form (32-column blocks, a row's long sums dealt over 4 partial
sums instead of 8) and the tile-pair form sum the products in other FP32
orders and are held, like every form, to the mixed form's tolerances
against the FP64 oracle: trajectories (t = 1.5) ||drho||_F <= 1e-6 and
max|dp| <= 1e-6 max p, steady states ||drho||_F <= 1e-6 and max|dp| <=
1e-7 max p.
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
FORMS = (Q.QPR_SPARSE_FORM_COLUMNS, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, Q.QPR_SPARSE_FORM_COLUMNS_GATHER,
         Q.QPR_SPARSE_FORM_TILES)
BITWISE = (Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT,)  # equal to COLUMNS


def _solver(g, omega, form, refresh=32, **kw):
    return Solver.from_edges(g, alpha=0.85, omega=omega, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                             sparse_form=form, ref_refresh=refresh, **kw)


def _close(got, ref, prel):
    p, pr = populations(got), populations(ref)
    assert np.linalg.norm(got - ref) <= 1e-6
    assert np.abs(p - pr).max() <= prel * pr.max()


def test_default_form_is_columns_where_it_fits():
    s = Solver.from_edges(graphs.heavy_tailed(300, 1), precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
    assert s.sparse_form == Q.QPR_SPARSE_FORM_COLUMNS
    big = Solver.from_edges(graphs.heavy_tailed(2000, 1), precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
    assert big.sparse_form == Q.QPR_SPARSE_FORM_COLUMNS_GATHER  # 2016 padded rows: the whole block does not fit
    plan = big.sparse_plan
    assert plan["splits"] >= 1 and plan["block_cols"] == 32 and plan["ctas"] == plan["splits"] * 2016 // 32
    small = Solver.from_edges(graphs.heavy_tailed(300, 1), precision=Q.QPR_MIXED,
                              backend=Q.QPR_BACKEND_SPARSE).sparse_plan
    assert small["block_cols"] == 16 and small["ctas"] == small["splits"] * 320 // 16 and small["smem"] > 0
    fp64 = Solver.from_edges(graphs.heavy_tailed(300, 1), backend=Q.QPR_BACKEND_SPARSE)
    assert fp64.sparse_form == 0


def test_largest_whole_block_against_oracle():
    # N = 1530 (1536 padded rows): the largest column block a CTA stages
    # whole (196 KB); the default plan picks the whole-block form there
    n = 1530
    g = graphs.heavy_tailed(n, 8)
    rho0 = graphs.random_density(n, 9, rank=2)
    ref = Oracle.from_edges(g, alpha=0.85, omega=0.6).evolve(rho0, 0.01, 20)
    s = Solver.from_edges(g, alpha=0.85, omega=0.6, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
    assert s.sparse_form == Q.QPR_SPARSE_FORM_COLUMNS and s.sparse_plan["block_cols"] == 16
    d = torch.from_numpy(rho0.copy()).to(DEV)
    s.evolve(d, 0.01, 20)
    got = d.cpu().numpy()
    _close(got, ref, 1e-6)
    assert np.abs(got - got.conj().T).max() == 0.0


@pytest.mark.parametrize("form", [Q.QPR_SPARSE_FORM_COLUMNS, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT])
def test_whole_block_forms_refused_where_they_do_not_fit(form):
    with pytest.raises(Q.QprError) as e:
        _solver(graphs.heavy_tailed(2000, 1), 0.8, form)
    assert e.value.status == Q.QPR_E_ARG


@pytest.mark.parametrize("n,omega,refresh", [(33, 0.8, 32), (200, 0.2, 7), (300, 0.8, 32), (520, 0.5, 16)])
def test_forms_trajectory(n, omega, refresh):
    g = graphs.heavy_tailed(n, 5)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.random_density(n, 4, rank=3)
    ref = o.evolve(rho0, 0.01, 150)
    got = {}
    for form in FORMS:
        s = _solver(g, omega, form, refresh)
        assert s.sparse_form == form
        d = torch.from_numpy(rho0.copy()).to(DEV)
        s.evolve(d, 0.01, 150)
        got[form] = d.cpu().numpy()
        _close(got[form], ref, 1e-6)
        assert np.abs(got[form] - got[form].conj().T).max() == 0.0
    for form in BITWISE:
        np.testing.assert_array_equal(got[form], got[Q.QPR_SPARSE_FORM_COLUMNS])


@pytest.mark.parametrize("n,omega", [(150, 0.8), (400, 0.3)])
def test_forms_steady_state(n, omega):
    g = graphs.heavy_tailed(n, 6)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.maximally_mixed(n)
    ref, steps_ref, _, _ = o.steady_state(rho0, 0.01, 1e-8, 200000)
    stats, states = {}, {}
    for form in FORMS:
        s = _solver(g, omega, form)
        d = torch.from_numpy(rho0.copy()).to(DEV)
        st = s.steady_state(d, 0.01, 1e-8, 200000)
        assert st["converged"] == 1 and st["residual"] < 1e-8
        assert abs(st["residual"] - o.residual(d.cpu().numpy())) <= 1e-12
        assert abs(st["steps"] - steps_ref) <= 1
        stats[form], states[form] = st, d.cpu().numpy()
        _close(states[form], ref, 1e-7)
    a = Q.QPR_SPARSE_FORM_COLUMNS
    for b in BITWISE:
        assert stats[a]["steps"] == stats[b]["steps"] and stats[a]["residual"] == stats[b]["residual"]
        np.testing.assert_array_equal(states[a], states[b])


def test_persistent_form_stops_at_max_steps():
    g = graphs.heavy_tailed(120, 7)
    s = _solver(g, 0.8, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, refresh=16)
    d = torch.from_numpy(graphs.maximally_mixed(120)).to(DEV)
    with pytest.raises(Q.QprError) as e:
        s.steady_state(d, 0.01, 1e-13, 45)
    assert e.value.status == Q.QPR_E_NOT_CONVERGED
    ref = Oracle.from_edges(g, alpha=0.85, omega=0.8).evolve(graphs.maximally_mixed(120), 0.01, 45)
    _close(d.cpu().numpy(), ref, 1e-6)


@pytest.fixture(scope="module")
def large_case():
    n, omega = 2000, 0.8
    g = graphs.heavy_tailed(n, 5)
    rho0 = graphs.random_density(n, 4, rank=3)
    ref = Oracle.from_edges(g, alpha=0.85, omega=omega).evolve(rho0, 0.01, 40)
    return g, omega, rho0, ref


@pytest.mark.parametrize("form", [Q.QPR_SPARSE_FORM_COLUMNS_GATHER, Q.QPR_SPARSE_FORM_TILES])
def test_large_n_trajectory(large_case, form):
    # N = 2000 (2016 padded rows), beyond the whole-block form
    g, omega, rho0, ref = large_case
    s = _solver(g, omega, form)
    assert s.sparse_form == form
    d = torch.from_numpy(rho0.copy()).to(DEV)
    s.evolve(d, 0.01, 40)
    got = d.cpu().numpy()
    _close(got, ref, 1e-6)
    assert np.abs(got - got.conj().T).max() == 0.0


def test_grid_barrier_timeout_is_reported_and_context_stays_usable():
    # test_fault makes every grid barrier of the persistent form wait for one
    # arrival more than its grid makes: no barrier completes, every CTA's
    # bounded wait gives up after its time limit (about a second), sets the
    # error flag and leaves the kernel. The host reads the flag and returns
    # QPR_E_TIMEOUT; no CUDA error occurs, so the context is not poisoned.
    import time
    g = graphs.heavy_tailed(120, 7)
    s = _solver(g, 0.8, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, refresh=16, test_fault=1)
    d = torch.from_numpy(graphs.maximally_mixed(120)).to(DEV)
    t = time.perf_counter()
    with pytest.raises(Q.QprError) as e:
        s.steady_state(d, 0.01, 1e-8, 1000)
    assert e.value.status == Q.QPR_E_TIMEOUT
    assert time.perf_counter() - t < 60.0
    # the same context still serves calls that need no grid barrier
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    rho = graphs.random_density(120, 3, rank=2)
    assert abs(s.residual(torch.from_numpy(rho).to(DEV)) - o.residual(rho)) <= 1e-12
    # and the device serves a context without the fault
    ok = _solver(g, 0.8, Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, refresh=16)
    d.copy_(torch.from_numpy(graphs.maximally_mixed(120)))
    st = ok.steady_state(d, 0.01, 1e-8, 200000)
    assert st["converged"] == 1
