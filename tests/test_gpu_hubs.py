"""Classical PageRank and hub classes through the C ABI (qpr_pagerank,
qpr_hub_classes) against the oracle.

The main text compares the quantum PageRank populations of the airline
network with the classical PageRank and counts main hubs (p > c/N) and
secondary hubs (1/N < p <= c/N), c = 10. qpr_pagerank is checked against
the oracle's power iteration on its own Google matrix (both dangling modes)
and against the omega = 1 steady-state populations of the oracle's RK4; hub
classes are integer decisions taken in FP64 on the same inputs on both sides,
so they must agree exactly, including on values equal to the thresholds.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle, superop
from oracle.cpu import hub_classes, populations
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n,seed,dangling", [(922, 1, Q.QPR_DANGLING_F), (300, 5, Q.QPR_DANGLING_UNIFORM),
                                             (2, 0, Q.QPR_DANGLING_F), (2000, 3, Q.QPR_DANGLING_F)])
def test_pagerank_matches_oracle_power_iteration(n, seed, dangling):
    g = graphs.heavy_tailed(n, seed) if n > 2 else graphs.erdos_renyi(2, 0.5, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, dangling=dangling)
    pi = s.pagerank(tol=1e-15, max_iter=100000)
    _, _, G, _ = Oracle.from_edges(g, alpha=0.85, omega=0.8, dangling=dangling).operators()
    ref = superop.stationary_by_power_iteration(G)
    assert abs(pi.sum() - 1.0) <= 1e-13
    assert np.abs(pi - ref).max() <= 1e-13 * max(1.0, ref.max() * n)
    # device output buffer
    d = torch.zeros(n, dtype=torch.float64, device=DEV)
    s.pagerank(tol=1e-15, out=d)
    np.testing.assert_array_equal(d.cpu().numpy(), pi)


def test_pagerank_is_the_omega1_steady_state():
    g = graphs.heavy_tailed(150, 2)
    s = Solver.from_edges(g, alpha=0.85, omega=1.0)
    pi = s.pagerank(tol=1e-15)
    o = Oracle.from_edges(g, alpha=0.85, omega=1.0)
    y, _, _, _ = o.steady_state(graphs.maximally_mixed(150), 0.01, 1e-12, 400000)
    np.testing.assert_allclose(pi, populations(y), rtol=0, atol=1e-10)


def test_pagerank_not_converged_is_reported():
    g = graphs.heavy_tailed(200, 4)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8)
    with pytest.raises(Q.QprError) as e:
        s.pagerank(tol=1e-15, max_iter=3)
    assert e.value.status == Q.QPR_E_NOT_CONVERGED


def test_hub_classes_match_oracle_on_qpr_and_pagerank():
    g = graphs.heavy_tailed(922, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED)
    rho = torch.from_numpy(graphs.maximally_mixed(922)).to(DEV)
    s.steady_state(rho, 0.01, 1e-8, 100000)
    p = s.populations(rho)
    for vec in (p, s.pagerank(tol=1e-15)):
        cls, counts = s.hub_classes(vec, 10.0)
        ref = hub_classes(vec, 10.0)
        np.testing.assert_array_equal(cls, ref)
        np.testing.assert_array_equal(counts, np.bincount(ref, minlength=3))
        # device input
        cls_d, counts_d = s.hub_classes(torch.from_numpy(vec).to(DEV), 10.0)
        np.testing.assert_array_equal(cls_d, ref)


def test_hub_classes_threshold_sides():
    # values exactly at 1/N and c/N: 1/N is not a hub, c/N is a secondary hub
    n = 40
    g = graphs.heavy_tailed(n, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8)
    p = np.full(n, 0.5 / n)
    p[0], p[1], p[2], p[3] = 1.0 / n, 10.0 / n, np.nextafter(10.0 / n, 1.0), np.nextafter(1.0 / n, 1.0)
    cls, counts = s.hub_classes(p, 10.0)
    assert list(cls[:4]) == [0, 1, 2, 1]
    np.testing.assert_array_equal(cls, hub_classes(p, 10.0))
    assert list(counts) == [n - 3, 2, 1]
    with pytest.raises(Q.QprError) as e:
        s.hub_classes(p, 0.5)
    assert e.value.status == Q.QPR_E_ARG
