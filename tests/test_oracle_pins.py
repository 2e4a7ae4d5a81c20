"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each test ties the oracle to something other than itself: hand-worked
operator values (tests/golden), the N^2 x N^2 superoperator built from the
N^2 jump operators with the Kronecker index formula (Eq. 2, Eq. 3), the exact
RK4 amplification of a linear ODE, closed forms at omega = 0 and omega = 1,
power iteration, and invariants of a density matrix.
"""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, superop
from oracle.cpu import OracleError, hub_classes, populations, prepare, ranking
from paper_2003_04930_gb300 import graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_graph():
    with open(os.path.join(GOLDEN, "operators_n4.json")) as f:
        gd = json.load(f)
    e = np.array(gd["edges_src_dst_w"], dtype=np.float64)
    return gd, e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), e[:, 2]


@pytest.mark.parametrize("h_diag", [0, 1])
@pytest.mark.parametrize("dangling", [0, 1])
def test_operators_match_hand_worked_example(h_diag, dangling):
    gd, src, dst, w = _golden_graph()
    o = Oracle(gd["n"], src, dst, w, alpha=gd["alpha"], omega=0.5, h_diag=h_diag, dangling=dangling)
    A, H, G, c = o.operators()
    np.testing.assert_array_equal(A, np.array(gd["A"]))
    Hx = np.array(gd["H_zero_diag"], dtype=np.float64)
    if h_diag == 1:
        Hx[np.diag_indices(4)] = gd["H_neg_outdeg_diag"]
    np.testing.assert_array_equal(H, Hx)
    Gx = np.array(gd["G_dangling_F"])
    if dangling == 1:
        Gx[:, 3] = gd["G_dangling_uniform_col3"]
    np.testing.assert_allclose(G, Gx, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c, np.ones(4), rtol=0, atol=1e-15)


def test_rhs_hand_worked_example():
    gd, src, dst, w = _golden_graph()
    o = Oracle(gd["n"], src, dst, w, alpha=gd["alpha"], omega=1.0)
    f = o.rhs(np.eye(4, dtype=np.complex128) / 4)
    np.testing.assert_allclose(np.diag(f).real, gd["rhs_maximally_mixed_omega1_diag"], atol=1e-15)
    off = f - np.diag(np.diag(f))
    assert np.abs(off).max() == 0.0
    assert np.abs(np.diag(f).imag).max() == 0.0


def test_invalid_inputs_rejected():
    src = np.array([0, 1]); dst = np.array([1, 0])
    with pytest.raises(OracleError):
        Oracle(1, src[:0], dst[:0])  # n < 2
    with pytest.raises(OracleError):
        Oracle(3, src, dst, alpha=1.5)
    with pytest.raises(OracleError):
        Oracle(3, src, dst, omega=-0.1)
    with pytest.raises(OracleError):
        Oracle(3, np.array([0, 3]), dst)  # index out of range
    with pytest.raises(OracleError):
        Oracle(3, src, dst, np.array([1.0, -1.0]))  # negative weight
    with pytest.raises(OracleError):
        Oracle(3, src, dst, np.array([1.0, np.nan]))  # non-finite weight


def test_kron_index_formula_matches_library_kron():
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 5):
        a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        np.testing.assert_array_equal(superop.kron_eq3(a, b), np.kron(a, b))


def test_vectorisation_identity():
    # vec(A X B) = (B^T kron A) vec(X): the column-stacking convention
    rng = np.random.default_rng(6)
    n = 4
    a, x, b = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(3))
    lhs = superop.vec(a @ x @ b)
    rhs = superop.kron_eq3(b.T, a) @ superop.vec(x)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


CASES = [
    # (n, p, seed, alpha, omega, h_diag, dangling)
    (5, 0.4, 1, 0.85, 0.8, 0, 0),
    (6, 0.3, 2, 0.85, 0.3, 1, 0),
    (7, 0.2, 3, 0.6, 0.5, 0, 1),
    (8, 0.25, 4, 0.85, 0.0, 0, 0),
    (8, 0.25, 4, 0.85, 1.0, 1, 1),
    (6, 0.0, 9, 0.85, 0.7, 0, 0),  # no links at all: every column dangles
]


@pytest.mark.parametrize("case", CASES)
def test_rhs_equals_superoperator_from_jump_operators(case):
    n, p, seed, alpha, omega, hd, dg = case
    g = graphs.erdos_renyi(n, p, seed)
    w = np.random.default_rng(seed + 100).lognormal(0, 1, g.m)
    o = Oracle(n, g.src, g.dst, w, alpha=alpha, omega=omega, h_diag=hd, dangling=dg)
    A, H, G, c = o.operators()
    lsup = superop.superoperator(H, G, omega)
    for s in range(3):
        rho = graphs.random_hermitian(n, 10 * seed + s)
        f_or = o.rhs(rho)
        f_su = superop.unvec(lsup @ superop.vec(rho), n)
        np.testing.assert_allclose(f_or, f_su, rtol=0, atol=1e-13 * max(1.0, np.abs(f_su).max()))
        # residual is the Frobenius norm of f over all N^2 entries
        assert abs(o.residual(rho) - np.linalg.norm(f_su)) <= 1e-13 * max(1.0, np.linalg.norm(f_su))


def test_rhs_is_trace_free_and_hermitian():
    g = graphs.heavy_tailed(40, 7)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.4)
    rho = graphs.random_density(40, 3)
    f = o.rhs(rho)
    assert abs(np.trace(f)) < 1e-13
    assert np.abs(f - f.conj().T).max() < 1e-13


@pytest.fixture(scope="module")
def config1():
    """The 16-node directed ER case: p = 0.25, seed 0, unit weights,
    alpha = 0.85, omega = 0.8, rho0 = I/N."""
    g = graphs.erdos_renyi(16, 0.25, 0)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    A, H, G, c = o.operators()
    lsup = superop.superoperator(H, G, 0.8)
    return g, o, H, G, lsup


def test_rk4_trajectory_equals_amplification_power(config1):
    # 10^4 RK4 steps of dt = 0.01 (t = 100) from I/N are exactly R(dt L)^n rho0
    g, o, H, G, lsup = config1
    rho0 = graphs.maximally_mixed(16)
    y = o.evolve(rho0, 0.01, 10000)
    ye, cond = superop.rk4_by_eigendecomposition(lsup, rho0, 0.01, 10000)
    assert cond < 1e4
    assert np.abs(y - ye).max() < 1e-11
    yp = superop.rk4_by_matrix_power(lsup, rho0, 0.01, 10000)
    assert np.abs(y - yp).max() < 1e-11


def test_rk4_fourth_order_convergence_to_exponential(config1):
    g, o, H, G, lsup = config1
    rho0 = graphs.random_density(16, 11, rank=1)
    t = 2.0
    exact = superop.exact_solution(lsup, rho0, t)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        y = o.evolve(rho0, dt, int(round(t / dt)))
        errs.append(np.abs(y - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, errs


def test_steady_state_equals_null_vector(config1):
    g, o, H, G, lsup = config1
    rss, s0, s1 = superop.null_state(lsup)
    assert s0 < 1e-12 and s1 > 1e-3  # one-dimensional null space
    y, steps, r, st = o.steady_state(graphs.maximally_mixed(16), 0.01, 1e-12, 200000)
    assert st == 0 and r < 1e-12
    assert np.abs(y - rss).max() < 1e-10
    # first step index below tol: the one before must not be
    y2, steps2, r2, st2 = o.steady_state(graphs.maximally_mixed(16), 0.01, 1e-12, steps - 1)
    assert st2 != 0 and r2 >= 1e-12


def test_omega1_populations_equal_classical_pagerank():
    g = graphs.heavy_tailed(24, 3)
    o = Oracle.from_edges(g, alpha=0.85, omega=1.0)
    A, H, G, c = o.operators()
    pstat = superop.stationary_by_power_iteration(G)
    y, steps, r, st = o.steady_state(graphs.random_density(24, 4), 0.01, 1e-11, 200000)
    assert st == 0
    np.testing.assert_allclose(populations(y), pstat, rtol=0, atol=1e-11)


def test_omega1_coherences_decay_by_rk4_factor():
    # at omega = 1 with c = 1 every coherence obeys d rho_ab/dt = -rho_ab
    g = graphs.erdos_renyi(12, 0.3, 8)
    o = Oracle.from_edges(g, alpha=0.85, omega=1.0)
    rho0 = prepare(graphs.random_density(12, 9))
    n = 300
    y = o.evolve(rho0, 0.01, n)
    off = ~np.eye(12, dtype=bool)
    factor = superop.rk4_amplification(-0.01) ** n
    np.testing.assert_allclose(y[off], factor * rho0[off], rtol=1e-12, atol=1e-15)


def test_omega0_purity_follows_rk4_amplification():
    # at omega = 0, in the eigenbasis of H, rho'_ab is multiplied by
    # R(-i dt (E_a - E_b)) every step: purity follows in closed form
    g = graphs.heavy_tailed(20, 5)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.0)
    A, H, G, c = o.operators()
    rho0 = graphs.random_density(20, 6, rank=1)
    dt, n = 0.01, 500
    y = o.evolve(rho0, dt, n)
    E, U = np.linalg.eigh(H)
    r0 = U.T @ rho0 @ U
    amp = np.abs(superop.rk4_amplification(-1j * dt * (E[:, None] - E[None, :]))) ** (2 * n)
    purity_pred = float(np.sum(np.abs(r0) ** 2 * amp))
    purity = float(np.real(np.trace(y @ y)))
    assert abs(purity - purity_pred) < 1e-12
    assert purity <= 1.0 + 1e-14
    # and the maximally mixed state is stationary at omega = 0
    assert np.abs(o.rhs(graphs.maximally_mixed(20))).max() == 0.0


def test_sign_of_H_leaves_populations_unchanged():
    g = graphs.heavy_tailed(10, 12)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.5)
    A, H, G, c = o.operators()
    r1, _, _ = superop.null_state(superop.superoperator(H, G, 0.5))
    r2, _, _ = superop.null_state(superop.superoperator(-H, G, 0.5))
    np.testing.assert_allclose(np.diag(r1).real, np.diag(r2).real, atol=1e-12)
    np.testing.assert_allclose(r1, r2.conj(), atol=1e-12)


@pytest.mark.parametrize("n,omega", [(16, 0.8), (64, 0.2)])
def test_density_matrix_invariants_along_trajectory(n, omega):
    g = graphs.heavy_tailed(n, 21)
    o = Oracle.from_edges(g, alpha=0.85, omega=omega)
    y = graphs.random_density(n, 22, rank=2)
    for _ in range(4):
        y = o.evolve(y, 0.01, 25)
        assert abs(np.trace(y).real - 1.0) < 1e-13
        assert np.abs(y - y.conj().T).max() == 0.0
        assert np.linalg.eigvalsh(y).min() > -1e-10


def test_rk4_stability_half_disk():
    # |R(z)| <= 1 on the left half-disk of radius 2.5, the region the solver's
    # step-size check relies on
    r = np.linspace(0, 2.5, 251)[:, None]
    th = np.linspace(np.pi / 2, 3 * np.pi / 2, 361)[None, :]
    z = r * np.exp(1j * th)
    assert np.abs(superop.rk4_amplification(z)).max() <= 1.0 + 1e-12
    # and it fails just outside the imaginary-axis limit 2*sqrt(2)
    assert abs(superop.rk4_amplification(2.9j)) > 1.0


def test_populations_ranking_hubs():
    p = np.array([0.05, 0.3, 0.05, 0.6])
    np.testing.assert_array_equal(ranking(p), [3, 1, 0, 2])
    # N = 4, c = 2: secondary 1/4 < p <= 1/2, main p > 1/2
    np.testing.assert_array_equal(hub_classes(p, c=2.0), [0, 1, 0, 2])
    rho = np.diag(p).astype(np.complex128)
    np.testing.assert_array_equal(populations(rho), p)


def test_prepare_hermitises_and_normalises():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5)) + 5 * np.eye(5)
    y = prepare(x)
    h = 0.5 * (x + x.conj().T)
    np.testing.assert_allclose(y, h / np.trace(h).real, atol=1e-15)
