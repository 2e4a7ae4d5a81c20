"""Seeded synthetic graph and state generators.

This module produces inputs only: edge lists and initial density matrices.
It holds none of the solver's arithmetic (no Hamiltonian, no Google matrix,
no Lindblad right-hand side), so both the CUDA path and the CPU oracle can
consume its output without sharing any of the method's code.

The paper's own workload is the 922-airport USA airline network (Sec. "USA
airline network", Fig. 2), which is not distributed with the paper. The
generators below stand in for it: a directed Erdos-Renyi graph for the small
case and a heavy-tailed preferential-attachment graph (power-law out-degrees,
lognormal weights) for the airline-sized and larger cases.

Edge convention: an edge is (src, dst, w) and means a link src -> dst.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class EdgeList:
    """A weighted directed edge list on nodes 0..n-1 (link src -> dst)."""

    n: int
    src: np.ndarray  # int64 [m]
    dst: np.ndarray  # int64 [m]
    w: np.ndarray  # float64 [m]

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def erdos_renyi(n: int, p: float, seed: int) -> EdgeList:
    """Directed Erdos-Renyi graph with unit weights.

    Draw order: one ``random((n, n))`` matrix U from ``default_rng(seed)``;
    the link j -> i exists when U[i, j] < p and i != j. Edges are listed in
    row-major order of (i, j).
    """
    rng = np.random.default_rng(seed)
    u = rng.random((n, n))
    mask = u < p
    np.fill_diagonal(mask, False)
    dst, src = np.nonzero(mask)
    return EdgeList(n, src.astype(np.int64), dst.astype(np.int64),
                    np.ones(src.shape[0], dtype=np.float64))


def powerlaw_out_degrees(n: int, gamma: float, mean_deg: float,
                         rng: np.random.Generator) -> np.ndarray:
    """Out-degrees from a discrete power law P(d) ~ d^-gamma.

    Continuous Pareto samples x >= 1 with density ~ x^-gamma are rescaled so
    that their sample mean is ``mean_deg``, rounded, and clipped to [1, n-1].
    """
    u = rng.random(n)
    x = (1.0 - u) ** (-1.0 / (gamma - 1.0))
    d = np.rint(x * (mean_deg / x.mean())).astype(np.int64)
    return np.clip(d, 1, n - 1)


def heavy_tailed(n: int, seed: int, gamma: float = 2.2, mean_deg: float = 8.0,
                 sigma: float = 1.0) -> EdgeList:
    """Heavy-tailed preferential-attachment digraph with lognormal weights.

    Draw order from ``default_rng(seed)``:
      1. ``n`` uniforms for the out-degrees (see ``powerlaw_out_degrees``);
      2. for each source node j = 0..n-1 in order, ``d_j`` distinct targets
         (never j) drawn without replacement with probability proportional to
         (in-degree + 1) of the targets at that moment; in-degrees are updated
         after node j's targets are chosen;
      3. one lognormal(0, sigma) weight per edge, in edge order.
    No self-loops and no duplicate (src, dst) pairs are produced.
    """
    rng = np.random.default_rng(seed)
    deg = powerlaw_out_degrees(n, gamma, mean_deg, rng)
    indeg = np.zeros(n, dtype=np.float64)
    srcs = []
    dsts = []
    for j in range(n):
        wgt = indeg + 1.0
        wgt[j] = 0.0
        prob = wgt / wgt.sum()
        tgt = rng.choice(n, size=int(deg[j]), replace=False, p=prob)
        srcs.append(np.full(tgt.shape[0], j, dtype=np.int64))
        dsts.append(tgt.astype(np.int64))
        indeg[tgt] += 1.0
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    w = rng.lognormal(0.0, sigma, size=src.shape[0])
    return EdgeList(n, src, dst, w.astype(np.float64))


def batch_specs(count: int = 512, seed: int = 2, n_lo: int = 32, n_hi: int = 1024,
                omega_lo: float = 0.1, omega_hi: float = 0.95):
    """Sizes, omegas and graph seeds of a batch of independent problems.

    From ``default_rng(seed)``: ``count`` integers N ~ U[n_lo, n_hi], then
    ``count`` omegas ~ U[omega_lo, omega_hi]. Graph g uses seed 1000 + g.
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    omegas = rng.uniform(omega_lo, omega_hi, size=count)
    return [(int(ns[g]), float(omegas[g]), 1000 + g) for g in range(count)]


def maximally_mixed(n: int) -> np.ndarray:
    """rho0 = I/N as an n x n complex128 array."""
    return np.eye(n, dtype=np.complex128) / n


def random_density(n: int, seed: int, rank: int | None = None) -> np.ndarray:
    """A random density matrix (Hermitian, PSD, unit trace), complex128.

    rho = W W^dagger / tr(W W^dagger) with W an n x rank complex Gaussian
    matrix drawn from ``default_rng(seed)`` (real parts first, then
    imaginary parts). ``rank=1`` gives a pure state.
    """
    rng = np.random.default_rng(seed)
    r = n if rank is None else rank
    wr = rng.standard_normal((n, r))
    wi = rng.standard_normal((n, r))
    wm = wr + 1j * wi
    rho = wm @ wm.conj().T
    rho = 0.5 * (rho + rho.conj().T)
    return rho / np.trace(rho).real


def random_hermitian(n: int, seed: int) -> np.ndarray:
    """A random Hermitian (not necessarily PSD) complex128 matrix."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (a + a.conj().T)
