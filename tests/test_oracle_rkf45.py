"""Pins of the oracle's adaptive RKF45 (Supplementary Note 2, Eq. S10 - S13).

Nothing here retypes the tableau. The pins are properties the printed scheme
has only when every coefficient is right:
  * one attempt's fourth-order solution y_{k+1} (Eq. S11) has local error
    O(h^5) against the exact exp(h L) y_k, and the fifth-order z_{k+1}
    (Eq. S12) O(h^6): halving h divides the errors by about 32 and 64 (with
    the printed 4101 instead of 4104, or any wrong stage coefficient, the
    weights no longer sum to one or an order condition fails and the ratio
    collapses towards 2);
  * the discrepancy |z - y| therefore scales as h^5;
  * for the linear ODE rho' = L rho every RK scheme preserves the trace and
    Hermiticity of the state, and the accepted trajectory of the adaptive
    loop stays within the tolerance it controls: the error against the exact
    exp(L t) rho_0 is at most of order step_tol * t, and every accepted
    attempt had |z - y| <= step_tol * h;
  * a fourth-order method under per-unit-step error control takes steps
    h ~ step_tol^(1/4): dividing step_tol by 16 doubles the number of steps;
  * with the step cap at the stability estimate the loop reaches the steady
    state (the null vector of the superoperator) like fixed-step RK4; where
    the coherences are weakly damped (omega = 0.5) the fourth-order
    propagated solution stalls and the fifth-order alternative converges.
"""
import numpy as np
import pytest

from oracle import Oracle, superop
from paper_2003_04930_gb300 import graphs


@pytest.fixture(scope="module")
def config1():
    g = graphs.erdos_renyi(16, 0.25, 0)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    A, H, G, c = o.operators()
    lsup = superop.superoperator(H, G, 0.8)
    hmax = 2.5 / ((1 - 0.8) * (np.linalg.eigvalsh(H)[-1] - np.linalg.eigvalsh(H)[0]) + 2 * 0.8 * c.max())
    return g, o, lsup, hmax


def test_embedded_pair_orders(config1):
    g, o, lsup, _ = config1
    rho0 = graphs.random_density(16, 3, rank=2)
    e4, e5, disc = [], [], []
    for h in (0.4, 0.2, 0.1):
        y4, z5, d = o.rkf45_step(rho0, h)
        ex = superop.exact_solution(lsup, rho0, h)
        e4.append(np.abs(y4 - ex).max())
        e5.append(np.abs(z5 - ex).max())
        disc.append(d)
        assert d == pytest.approx(np.abs(z5 - y4).max(), rel=1e-12)
    for a, b in zip(e4, e4[1:]):
        assert 24.0 < a / b < 40.0, e4   # local error O(h^5)
    for a, b in zip(e5, e5[1:]):
        assert 48.0 < a / b < 80.0, e5   # local error O(h^6)
    for a, b in zip(disc, disc[1:]):
        assert 24.0 < a / b < 40.0, disc


def test_single_attempt_preserves_trace_and_hermiticity(config1):
    g, o, lsup, _ = config1
    rho0 = graphs.random_density(16, 5, rank=3)
    y4, z5, _ = o.rkf45_step(rho0, 0.1)
    for y in (y4, z5):
        assert abs(np.trace(y) - 1.0) < 1e-14
        assert np.abs(y - y.conj().T).max() < 1e-15


def test_adaptive_trajectory_within_controlled_tolerance(config1):
    g, o, lsup, hmax = config1
    rho0 = graphs.random_density(16, 7, rank=1)
    t_end = 3.0
    exact = superop.exact_solution(lsup, rho0, t_end)
    for tol, order in ((1e-5, 4), (1e-7, 4), (1e-7, 5)):
        out = o.rkf45(rho0, 0.01, tol, hmax, t_end=t_end, history=True, order=order)
        assert out["t"] == t_end and out["status"] == 0
        hist = out["history"]
        acc = hist[hist[:, 4] == 1]
        assert len(acc) == out["accepted"] and len(hist) == out["accepted"] + out["rejected"]
        assert np.all(acc[:, 2] <= tol * acc[:, 1])          # accepted: discrepancy <= Tol h
        rej = hist[hist[:, 4] == 0]
        assert np.all(rej[:, 2] > tol * rej[:, 1])
        assert np.all(hist[:, 1] <= hmax * (1 + 1e-15))
        assert abs(np.sum(acc[:, 1]) - t_end) < 1e-12          # the accepted steps tile [0, t_end]
        err = np.abs(out["rho"] - exact).max()
        assert err <= tol * t_end, (tol, err)


def test_step_count_scales_as_tolerance_to_the_quarter():
    # a transient whose step size is set by accuracy, not by the cap (no cap,
    # t = 1): with per-unit-step control the discrepancy ~ C h^5 is held near
    # Tol h, so h ~ Tol^(1/4) and the step count doubles when Tol / 16
    g = graphs.heavy_tailed(16, 2)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.8)
    rho0 = graphs.random_density(16, 9, rank=1)
    steps = []
    for tol in (1e-7, 1e-7 / 16, 1e-7 / 256):
        out = o.rkf45(rho0, 1e-3, tol, 10.0, t_end=1.0)
        steps.append(out["accepted"])
    for a, b in zip(steps, steps[1:]):
        assert 1.8 < b / a < 2.2, steps


@pytest.mark.parametrize("order", [4, 5])
def test_steady_state_equals_null_vector(config1, order):
    g, o, lsup, hmax = config1
    rho_ss, s_min, s2 = superop.null_state(lsup)
    out = o.rkf45(graphs.maximally_mixed(16), 0.01, 1e-4, hmax, resid_tol=1e-12, max_steps=100000, order=order)
    assert out["status"] == 0 and out["residual"] < 1e-12
    # two states with residual < r differ by at most about r / (second singular value)
    assert np.abs(out["rho"] - rho_ss).max() <= 1e-12 / s2 * 10
    # and it needs fewer steps than fixed-step RK4 at dt = 0.01
    _, rk4_steps, _, _ = o.steady_state(graphs.maximally_mixed(16), 0.01, 1e-12, 10**6)
    assert out["accepted"] < rk4_steps


def test_fifth_order_propagation_reaches_steady_state_where_fourth_stalls():
    # both propagated solutions are slightly anti-damping near the imaginary
    # axis (|P4(iy)| up to 1.03 and |P5(iy)| up to 1.004 for y < ~2.3); at
    # omega = 0.5 the coherences' damping omega h does not offset P4's, and the
    # residual stalls, while the fifth-order solution converges
    g = graphs.heavy_tailed(60, 6)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.5)
    A, H, G, c = o.operators()
    ev = np.linalg.eigvalsh(H)
    hmax = 2.5 / ((1 - 0.5) * (ev[-1] - ev[0]) + 2 * 0.5 * c.max())
    rho0 = graphs.maximally_mixed(60)
    four = o.rkf45(rho0, 0.01, 1e-6, hmax, resid_tol=1e-8, max_steps=4000, order=4)
    five = o.rkf45(rho0, 0.01, 1e-6, hmax, resid_tol=1e-8, max_steps=4000, order=5)
    assert four["status"] != 0 and four["residual"] > 1e-6
    assert five["status"] == 0 and five["residual"] < 1e-8


def test_invalid_arguments():
    g = graphs.erdos_renyi(8, 0.3, 1)
    o = Oracle.from_edges(g, alpha=0.85, omega=0.5)
    from oracle.cpu import OracleError
    for kw in (dict(h0=0.0), dict(step_tol=-1.0), dict(h_max=0.0)):
        args = dict(h0=0.01, step_tol=1e-6, h_max=0.1)
        args.update(kw)
        with pytest.raises(OracleError):
            o.rkf45(graphs.maximally_mixed(8), args["h0"], args["step_tol"], args["h_max"], t_end=1.0)
