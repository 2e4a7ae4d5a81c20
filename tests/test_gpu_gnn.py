"""Warm-start network on the GPU against its FP64 oracle, and the gain it
brings to the solver.

Tolerances: the GPU evaluates the same definition with FP32 activations and
accumulation (weights rounded to BF16 on both sides), so p_hat and the loss
agree to ~1e-6 relative and the gradient to ~1e-5 relative of its norm.
"""
import numpy as np
import pytest
import torch

from oracle import gnn as ognn
from paper_2003_04930_gb300 import Solver, graphs, warmstart
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _params(seed, scale=0.15):
    return (np.random.default_rng(seed).standard_normal(ognn.param_count()) * scale).astype(np.float32)


@pytest.mark.parametrize("n,omega,seed", [(40, 0.4, 3), (129, 0.9, 4), (300, 0.15, 5)])
def test_forward_and_gradient_match_oracle(n, omega, seed):
    g = graphs.heavy_tailed(n, seed)
    th = _params(seed)
    net = Q.Gnn(seed=1)
    net.set_params(th)
    np.testing.assert_array_equal(net.get_params(), th)
    p = np.random.default_rng(seed).random(n)
    p /= p.sum()
    l_ref, g_ref, ph_ref = ognn.loss_and_grad(th.astype(np.float64), n, g.src, g.dst, g.w, omega, 0.85, p)
    ph = net.predict(g, omega)
    np.testing.assert_allclose(ph, ph_ref, rtol=2e-5, atol=0)
    loss, grad = net.loss_grad(g, omega, p)
    assert abs(loss - l_ref) <= 1e-5 * abs(l_ref)
    err = np.linalg.norm(grad - g_ref) / np.linalg.norm(g_ref)
    assert err <= 2e-5, err
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    np.testing.assert_allclose(grad[big], g_ref[big], rtol=1e-3, atol=1e-5 * np.abs(g_ref).max())


def test_training_is_reproducible_and_reduces_loss():
    data = warmstart.make_dataset(warmstart.training_specs(16, n_lo=40, n_hi=120))
    nets = [Q.Gnn(seed=7) for _ in range(2)]
    losses = [net.train(data, epochs=15, batch=4, lr=3e-3, seed=11) for net in nets]
    np.testing.assert_array_equal(losses[0], losses[1])
    np.testing.assert_array_equal(nets[0].get_params(), nets[1].get_params())
    assert losses[0][-1] < losses[0][0]


def test_warm_start_saves_steps_and_keeps_the_answer():
    data = warmstart.make_dataset(warmstart.training_specs(48, n_lo=64, n_hi=256))
    net = Q.Gnn(seed=3)
    net.train(data, epochs=40, batch=8, lr=3e-3, seed=5)
    g = graphs.heavy_tailed(400, 7)  # not a training seed
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED)
    cold = torch.from_numpy(graphs.maximally_mixed(400)).to(DEV)
    st_cold = s.steady_state(cold, 0.01, 1e-8, 400000)
    p_hat = net.predict(g, 0.8)
    warm = torch.from_numpy(warmstart.warm_rho(p_hat)).to(DEV)
    st_warm = s.steady_state(warm, 0.01, 1e-8, 400000)
    assert st_warm["converged"] == 1
    assert st_warm["steps"] < st_cold["steps"], (st_warm["steps"], st_cold["steps"])
    # Two states that each pass resid < 1e-8 along different trajectories
    # differ by up to ~resid / gap, more than 1e-7 max p when max p ~ 1/N; the
    # cold and warm answers are compared after both are polished to 1e-11.
    s.steady_state(cold, 0.01, 1e-11, 400000)
    s.steady_state(warm, 0.01, 1e-11, 400000)
    a, b = cold.cpu().numpy(), warm.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-6
    pa, pb = np.real(np.diag(a)), np.real(np.diag(b))
    assert np.abs(pa - pb).max() <= 1e-7 * pa.max()


def test_shipped_network_saves_steps_at_n922():
    """The weights train_warmstart saved in the package (256 solver-generated
    steady states, seeds 10000+) on the N = 922 benchmark graph (seed 1)."""
    net = warmstart.load_network()
    assert net is not None
    g = graphs.heavy_tailed(922, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED)
    cold = torch.from_numpy(graphs.maximally_mixed(922)).to(DEV)
    st_cold = s.steady_state(cold, 0.01, 1e-8, 400000)
    warm = torch.from_numpy(warmstart.initial_state(net, g, 0.8)).to(DEV)
    st_warm = s.steady_state(warm, 0.01, 1e-8, 400000)
    assert st_warm["converged"] == 1 and st_warm["steps"] < st_cold["steps"], (st_warm["steps"], st_cold["steps"])
    s.steady_state(cold, 0.01, 1e-11, 400000)
    s.steady_state(warm, 0.01, 1e-11, 400000)
    pa, pb = np.real(np.diag(cold.cpu().numpy())), np.real(np.diag(warm.cpu().numpy()))
    assert np.abs(pa - pb).max() <= 1e-7 * pa.max()
