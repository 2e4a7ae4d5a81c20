"""Batched solver: every problem's result is bitwise the single-problem
mixed-form result (the batched kernels run the same per-tile and
per-problem device functions in the same order), and matches the FP64
oracle's steady state within the precision form's tolerance."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle.cpu import populations
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SPECS = [(32, 0.3, 1001), (50, 0.95, 1002), (97, 0.5, 1003), (150, 0.8, 1004), (200, 0.2, 1005), (64, 0.6, 1006)]


def _problems(host=False):
    out = []
    for n, om, seed in SPECS:
        g = graphs.heavy_tailed(n, seed)
        rho = graphs.maximally_mixed(n)
        out.append((g, om, rho.copy() if host else torch.from_numpy(rho).to(DEV)))
    return out


def test_batch_bitwise_equals_single_problem_solves():
    probs = _problems()
    st, stats = Q.batch_steady_state(probs, ref_refresh=16)
    assert st == Q.QPR_OK
    for (g, om, rho), s in zip(probs, stats):
        single = Solver.from_edges(g, alpha=0.85, omega=om, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                                   ref_refresh=16)
        r1 = torch.from_numpy(graphs.maximally_mixed(g.n)).to(DEV)
        s1 = single.steady_state(r1, 0.01, 1e-8, 400000)
        assert s["steps"] == s1["steps"] and s["converged"] == 1
        assert s["residual"] == s1["residual"]
        np.testing.assert_array_equal(rho.cpu().numpy(), r1.cpu().numpy())


def test_batch_matches_oracle_and_host_buffers():
    probs = _problems(host=True)
    st, stats = Q.batch_steady_state(probs)
    assert st == Q.QPR_OK
    for (g, om, rho), s in zip(probs, stats):
        o = Oracle.from_edges(g, alpha=0.85, omega=om)
        ref, steps, r, ost = o.steady_state(graphs.maximally_mixed(g.n), 0.01, 1e-8, 400000)
        assert ost == 0 and abs(s["steps"] - steps) <= 1
        p, pr = populations(rho), populations(ref)
        assert np.linalg.norm(rho - ref) <= 1e-6
        assert np.abs(p - pr).max() <= 1e-7 * pr.max()
        assert abs(s["residual"] - o.residual(rho)) <= 1e-12


def test_batch_max_steps():
    probs = _problems()
    st, stats = Q.batch_steady_state(probs, max_steps=40, check=False)
    assert st == Q.QPR_E_NOT_CONVERGED
    for (g, om, rho), s in zip(probs, stats):
        assert s["steps"] == 40 and s["converged"] == 0
        ref = Oracle.from_edges(g, alpha=0.85, omega=om).evolve(graphs.maximally_mixed(g.n), 0.01, 40)
        assert np.linalg.norm(rho.cpu().numpy() - ref) <= 1e-6


def test_batch_size_classes_and_tile_fallback_bitwise():
    # problems in both size classes of the batched SpMM (padded edge <= 512
    # and above) and one beyond the whole-block form (N = 1600: the tile-pair
    # form); omegas spread so problems retire at different blocks and the
    # captured lists are rebuilt on the way
    specs = [(100, 0.9, 2001), (300, 0.8, 2002), (600, 0.85, 2003), (900, 0.95, 2004), (1600, 0.9, 2005),
             (120, 0.4, 2006), (80, 0.7, 2007), (60, 0.95, 2008)]
    probs = []
    for n, om, seed in specs:
        g = graphs.heavy_tailed(n, seed)
        probs.append((g, om, torch.from_numpy(graphs.maximally_mixed(n)).to(DEV)))
    st, stats = Q.batch_steady_state(probs, ref_refresh=16)
    assert st == Q.QPR_OK
    for (g, om, rho), s in zip(probs, stats):
        form = Q.QPR_SPARSE_FORM_TILES if g.n > 1536 else Q.QPR_SPARSE_FORM_COLUMNS
        single = Solver.from_edges(g, alpha=0.85, omega=om, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                                   ref_refresh=16, sparse_form=form)
        r1 = torch.from_numpy(graphs.maximally_mixed(g.n)).to(DEV)
        s1 = single.steady_state(r1, 0.01, 1e-8, 400000)
        assert s["steps"] == s1["steps"] and s["converged"] == 1, g.n
        assert s["residual"] == s1["residual"]
        np.testing.assert_array_equal(rho.cpu().numpy(), r1.cpu().numpy())


def test_batch_tiny_problems_and_a_non_finite_start():
    # the smallest problems the method has (N = 2, 3: one padded 32 x 32 tile)
    # beside a regular one, and a problem whose start holds a NaN: the call
    # reports QPR_E_NONFINITE for the batch, that problem is not converged,
    # and the others are solved exactly as they are alone
    specs = [(2, 0.7, 2001), (3, 0.4, 2002), (140, 0.8, 2003), (90, 0.6, 2004)]
    probs = []
    for k, (n, om, seed) in enumerate(specs):
        g = graphs.erdos_renyi(n, 0.6, seed) if n < 10 else graphs.heavy_tailed(n, seed)
        rho = graphs.maximally_mixed(n)
        if k == 3:
            rho[1, 2] = np.nan
            rho[2, 1] = np.nan
        probs.append((g, om, torch.from_numpy(rho).to(DEV)))
    st, stats = Q.batch_steady_state(probs, check=False)
    assert st == Q.QPR_E_NONFINITE
    assert stats[3]["converged"] == 0
    for (g, om, rho), s in zip(probs[:3], stats[:3]):
        assert s["converged"] == 1
        single = Solver.from_edges(g, alpha=0.85, omega=om, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
        r1 = torch.from_numpy(graphs.maximally_mixed(g.n)).to(DEV)
        s1 = single.steady_state(r1, 0.01, 1e-8, 400000)
        assert s["steps"] == s1["steps"]
        np.testing.assert_array_equal(rho.cpu().numpy(), r1.cpu().numpy())
        ref, steps, _, _ = Oracle.from_edges(g, alpha=0.85, omega=om).steady_state(graphs.maximally_mixed(g.n),
                                                                                   0.01, 1e-8, 400000)
        assert np.abs(populations(rho.cpu().numpy()) - populations(ref)).max() <= 1e-7 * populations(ref).max()
