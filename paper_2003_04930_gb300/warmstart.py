"""Learned warm start: training data from the solver, training, rho0.

The network (``qpr.Gnn``) learns the steady-state populations p from graphs
whose steady states the batched solver itself computes; a solve then starts
from rho0 = diag(p_hat) instead of I/N. The solver's stop rule still decides
the result, so a poor prediction costs steps, never accuracy.
"""
from __future__ import annotations

import os

import numpy as np

from . import graphs
from . import qpr as Q


def training_specs(count: int, seed: int = 10000, n_lo: int = 64, n_hi: int = 2048, omega_lo: float = 0.1,
                   omega_hi: float = 0.95):
    """(N, omega, graph seed) of the training set: from default_rng(seed),
    `count` N ~ U[n_lo, n_hi] then `count` omega ~ U[omega_lo, omega_hi];
    graph i uses seed `seed + i` (disjoint from the evaluation seeds)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    om = rng.uniform(omega_lo, omega_hi, size=count)
    return [(int(ns[i]), float(om[i]), seed + i) for i in range(count)]


def make_dataset(specs, alpha=0.85, tol=1e-6, device="cuda:0"):
    """Steady states of the spec'd graphs from qpr_batch_steady_state (labels
    need about 1e-4 accuracy, so tol = 1e-6 is ample). Returns a list of
    (EdgeList, omega, p)."""
    import torch
    gs = [graphs.heavy_tailed(n, s) for n, om, s in specs]
    rhos = [torch.from_numpy(graphs.maximally_mixed(g.n)).to(device) for g in gs]
    Q.batch_steady_state([(g, om, r) for g, (n, om, s), r in zip(gs, specs, rhos)], alpha=alpha, tol=tol)
    return [(g, om, np.real(np.diag(r.cpu().numpy())).copy()) for g, (n, om, s), r in zip(gs, specs, rhos)]


def warm_rho(p_hat: np.ndarray) -> np.ndarray:
    """rho0 = diag(p_hat) (p_hat is positive and sums to one)."""
    return np.diag(np.asarray(p_hat, dtype=np.float64)).astype(np.complex128)


# A start with the right populations but no coherences helps only when the
# dissipator dominates: measured on the N = 922 workload, starting from the
# exact steady-state populations takes 1942 steps against 2226 from I/N at
# omega = 0.8, 3110 against 3129 at omega = 0.5, and 7875 against 7208 at
# omega = 0.2 (the coherent part must rebuild the coherences it was not
# given, and the populations move away meanwhile).
WARM_OMEGA_MIN = 0.5


TRAINED_PARAMS = os.path.join(os.path.dirname(__file__), "data", "warmstart_gnn.npy")


def load_network(path: str = TRAINED_PARAMS, device: int = -1):
    """The network with the parameters train_warmstart saved (None if the
    file is absent)."""
    if not os.path.exists(path):
        return None
    net = Q.Gnn(seed=0, device=device)
    net.set_params(np.load(path).astype(np.float32))
    return net


def initial_state(net, g, omega: float, alpha: float = 0.85) -> np.ndarray:
    """The solver's initial state: diag(p_hat) from the network when
    omega >= WARM_OMEGA_MIN, else the fallback I/N."""
    if net is None or omega < WARM_OMEGA_MIN:
        return graphs.maximally_mixed(g.n)
    return warm_rho(net.predict(g, omega, alpha))
