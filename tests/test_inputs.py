"""The seeded input generators follow the recipe the measurements state: the
heavy-tailed digraph (power-law out-degrees of mean about 8, targets without
self-loops or duplicates, lognormal(0, 1) weights), the batch of 512 problems
(N ~ U[32, 1024], omega ~ U[0.1, 0.95], graph seeds 1000 + g), the
Erdos-Renyi config-1 graph, and the density-matrix starts; every generator is
a pure function of its seed."""
import numpy as np
import pytest

from paper_2003_04930_gb300 import graphs


@pytest.mark.parametrize("n,seed", [(922, 1), (2048, 1)])
def test_heavy_tailed_recipe(n, seed):
    g = graphs.heavy_tailed(n, seed)
    assert g.n == n and g.src.dtype == np.int64 and g.dst.dtype == np.int64
    assert np.all((g.src >= 0) & (g.src < n) & (g.dst >= 0) & (g.dst < n))
    assert not np.any(g.src == g.dst)                               # no self-loops
    assert len(set(zip(g.src.tolist(), g.dst.tolist()))) == g.m    # no duplicates
    outdeg = np.bincount(g.src, minlength=n)
    assert outdeg.min() >= 1 and outdeg.max() <= n - 1
    assert 7.0 <= outdeg.mean() <= 9.0                              # rescaled to mean 8, then rounded and clipped
    assert outdeg.max() > 20 * np.median(outdeg)                    # heavy tail
    indeg = np.bincount(g.dst, minlength=n)
    assert indeg.max() > 3 * max(1.0, np.median(indeg))             # preferential attachment (in-degree + 1)
    assert np.all(g.w > 0.0)
    lw = np.log(g.w)
    assert abs(lw.mean()) < 0.05 and abs(lw.std() - 1.0) < 0.05     # lognormal(0, 1)


def test_generators_are_pure_functions_of_the_seed():
    a, b, c = graphs.heavy_tailed(300, 4), graphs.heavy_tailed(300, 4), graphs.heavy_tailed(300, 5)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.w, b.w)
    assert not (a.m == c.m and np.array_equal(a.src, c.src) and np.array_equal(a.dst, c.dst))
    assert np.array_equal(graphs.random_density(20, 3), graphs.random_density(20, 3))


def test_batch_recipe():
    specs = graphs.batch_specs(512)
    assert len(specs) == 512
    ns = np.array([s[0] for s in specs])
    oms = np.array([s[1] for s in specs])
    assert ns.min() >= 32 and ns.max() <= 1024
    assert oms.min() >= 0.1 and oms.max() <= 0.95
    assert [s[2] for s in specs] == [1000 + g for g in range(512)]
    assert specs == graphs.batch_specs(512)
    # roughly uniform: the quartiles of N and omega near those of U[32, 1024] and U[0.1, 0.95]
    assert np.allclose(np.percentile(ns, [25, 50, 75]), [280, 528, 776], atol=60)
    assert np.allclose(np.percentile(oms, [25, 50, 75]), [0.3125, 0.525, 0.7375], atol=0.06)


def test_config1_erdos_renyi():
    g = graphs.erdos_renyi(16, 0.25, 0)
    assert g.n == 16 and not np.any(g.src == g.dst) and np.all(g.w == 1.0)
    assert 30 <= g.m <= 90  # p = 0.25 of the 240 ordered pairs


@pytest.mark.parametrize("rank", [None, 1, 3])
def test_density_matrix_starts(rank):
    rho = graphs.random_density(12, 7, rank=rank)
    assert np.allclose(rho, rho.conj().T, atol=1e-15)
    assert abs(np.trace(rho).real - 1.0) < 1e-14
    ev = np.linalg.eigvalsh(rho)
    assert ev.min() > -1e-14
    assert np.sum(ev > 1e-12) == (12 if rank is None else rank)
    mm = graphs.maximally_mixed(5)
    assert np.allclose(mm, np.eye(5) / 5)
