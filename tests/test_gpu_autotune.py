"""The autotuner times real runs of the candidate configurations, caches
its choice (returned as is on the next call), and its choice runs: a solver
built from the result uses the chosen form and runs a step no slower than
the fixed rule's default configuration (within timing noise)."""
import time

import pytest
import torch

from paper_2003_04930_gb300 import graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu


def _ms_per_step(s, n, steps=256):
    rho = torch.from_numpy(graphs.maximally_mixed(n)).cuda()
    s.evolve(rho, 0.01, 32)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        t = time.perf_counter()
        s.evolve(rho, 0.01, steps)
        torch.cuda.synchronize()
        best = min(best, (time.perf_counter() - t) / steps * 1e3)
    return best


def test_autotune_chooses_and_caches(tmp_path):
    g = graphs.heavy_tailed(300, 1)
    cache = tmp_path / "tune.txt"
    r = Q.autotune(g, 0.8, cache_path=cache)
    assert r["backend"] in (Q.QPR_BACKEND_SPARSE, Q.QPR_BACKEND_DENSE)
    assert r["ref_refresh"] in (16, 32, 64) and r["ms_per_step"] > 0 and r["from_cache"] == 0
    line = cache.read_text().strip().split()
    assert len(line) == 6 and int(line[1]) == r["backend"] and int(line[2]) == r["ref_refresh"]
    assert int(line[4]) == r["sparse_form"] and int(line[5]) == r["row_splits"]
    r2 = Q.autotune(g, 0.8, cache_path=cache)
    assert r2["from_cache"] == 1 and {k: r2[k] for k in ("backend", "ref_refresh", "sparse_form", "row_splits")} \
        == {k: r[k] for k in ("backend", "ref_refresh", "sparse_form", "row_splits")}
    # the heavy-tailed graph has nnz(H) ~ 16 N: a sparse form wins
    assert r["backend"] == Q.QPR_BACKEND_SPARSE
    s = Q.Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, **Q.tuned_options(r))
    assert s.backend == r["backend"]
    if r["sparse_form"] != Q.QPR_SPARSE_FORM_AUTO:
        assert s.sparse_form == r["sparse_form"]


@pytest.mark.parametrize("n", [922, 2500])
def test_tuned_choice_not_slower_than_fixed_rule(n):
    g = graphs.heavy_tailed(n, 1)
    r = Q.autotune(g, 0.8)
    tuned = Q.Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, **Q.tuned_options(r))
    fixed = Q.Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED)
    t_tuned, t_fixed = _ms_per_step(tuned, n), _ms_per_step(fixed, n)
    print(f"N={n}: tuned {r} {t_tuned:.4f} ms/step, fixed rule {t_fixed:.4f} ms/step")
    assert t_tuned <= 1.10 * t_fixed
