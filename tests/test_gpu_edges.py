"""Degenerate cases of the method, on every stage form, against the FP64
oracle (150 RK4 steps from a random low-rank density matrix):

  * omega = 0: Eq. 1 without the dissipator, a unitary evolution under H,
    whose purity Tr rho^2 the exact flow conserves (the GPU's purity must
    follow the oracle's RK4 purity);
  * omega = 1: no coherent part, the classical random walk of G;
  * a graph without edges: H = 0 and every node dangles, so only the
    dissipator's uniform teleportation acts;
  * the smallest problems, N = 2 (one edge, one dangling node) and N = 3,
    which leave all but a few rows of every padded tile empty;
  * a star (every leaf links to the hub and the hub to every leaf): one row
    and one column of H with N - 1 nonzeros beside rows of one.

Tolerances: the FP64 forms at ||drho||_F <= 1e-11; the mixed forms at
their trajectory bounds (||drho||_F <= 1e-6, max|dp| <= 1e-6 max p); every
state exactly Hermitian with unit trace.
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
STEPS = 150

FORMS = {
    "fp64-sparse": dict(precision=Q.QPR_FP64, backend=Q.QPR_BACKEND_SPARSE),
    "fp64-dense": dict(precision=Q.QPR_FP64, backend=Q.QPR_BACKEND_DENSE),
    "mixed-columns": dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                          sparse_form=Q.QPR_SPARSE_FORM_COLUMNS, ref_refresh=16),
    "mixed-persistent": dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                             sparse_form=Q.QPR_SPARSE_FORM_COLUMNS_PERSISTENT, ref_refresh=16),
    "mixed-gather": dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                         sparse_form=Q.QPR_SPARSE_FORM_COLUMNS_GATHER, ref_refresh=16),
    "mixed-tiles": dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE, sparse_form=Q.QPR_SPARSE_FORM_TILES,
                        ref_refresh=16),
    "mixed-tc": dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_DENSE, ref_refresh=16),
}


def _star(n):
    leaves = np.arange(1, n, dtype=np.int64)
    hub = np.zeros(n - 1, dtype=np.int64)
    src = np.concatenate([leaves, hub])
    dst = np.concatenate([hub, leaves])
    return graphs.EdgeList(n, src, dst, np.ones(src.shape[0]))


CASES = {
    "omega0": (lambda: graphs.heavy_tailed(150, 4), 0.0),
    "omega1": (lambda: graphs.heavy_tailed(150, 4), 1.0),
    "no-edges": (lambda: graphs.erdos_renyi(40, 0.0, 0), 0.6),
    "n2": (lambda: graphs.EdgeList(2, np.array([0]), np.array([1]), np.array([1.0])), 0.8),
    "n3": (lambda: graphs.erdos_renyi(3, 0.6, 1), 0.5),
    "star": (lambda: _star(200), 0.8),
}


def _purity(r):
    return float(np.real(np.trace(r @ r)))


@pytest.mark.parametrize("case", sorted(CASES))
def test_degenerate_cases_on_every_form(case):
    make, omega = CASES[case]
    g = make()
    n = g.n
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    rho0 = graphs.random_density(n, 3, rank=min(2, n))
    probe = Solver.from_edges(g, alpha=0.85, omega=omega)
    dt = min(0.01, 0.9 * probe.max_stable_dt)
    probe.close()
    ref = o.evolve(rho0, dt, STEPS)
    for name, kw in FORMS.items():
        s = Solver.from_edges(g, alpha=0.85, omega=omega, **kw)
        d = torch.from_numpy(rho0.copy()).to(DEV)
        s.evolve(d, dt, STEPS)
        got = d.cpu().numpy()
        s.close()
        assert np.abs(got - got.conj().T).max() == 0.0, name
        assert abs(np.trace(got).real - 1.0) < 1e-13, name
        err = np.linalg.norm(got - ref)
        if name.startswith("fp64"):
            assert err <= 1e-11, (name, err)
        else:
            p, pr = populations(got), populations(ref)
            assert err <= 1e-6, (name, err)
            assert np.abs(p - pr).max() <= 1e-6 * pr.max(), name
        if omega == 0.0:
            # |Tr a^2 - Tr b^2| <= ||a - b||_F ||a + b||_F <= 2 ||a - b||_F (purity <= 1)
            bound = 2.0 * (1e-11 if name.startswith("fp64") else 1e-6)
            assert abs(_purity(got) - _purity(ref)) <= bound, name


@pytest.mark.parametrize("name", ["fp64-sparse", "mixed-columns", "mixed-gather"])
def test_smallest_problem_steady_state(name):
    # N = 2 with one link 0 -> 1: node 1 dangles and teleports uniformly
    g = graphs.EdgeList(2, np.array([0]), np.array([1]), np.array([1.0]))
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    rref, steps, _, _ = o.steady_state(graphs.maximally_mixed(2), 0.01, 1e-8, 100000)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, **FORMS[name])
    d = torch.from_numpy(graphs.maximally_mixed(2)).to(DEV)
    st = s.steady_state(d, 0.01, 1e-8, 100000)
    got = d.cpu().numpy()
    assert st["converged"] == 1 and st["residual"] < 1e-8
    assert abs(st["steps"] - steps) <= 1
    p, pr = populations(got), populations(rref)
    assert np.abs(p - pr).max() <= 1e-7 * pr.max()
