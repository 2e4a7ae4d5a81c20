"""The autotuner picks a configuration that runs, caches it, and the cached
choice is returned on the next call."""
import pytest

from paper_2003_04930_gb300 import graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu


def test_autotune_chooses_and_caches(tmp_path):
    g = graphs.heavy_tailed(300, 1)
    cache = tmp_path / "tune.txt"
    r = Q.autotune(g, 0.8, cache_path=cache)
    assert r["backend"] in (Q.QPR_BACKEND_SPARSE, Q.QPR_BACKEND_DENSE)
    assert r["ref_refresh"] in (8, 16, 32, 64) and r["ms_per_step"] > 0 and r["from_cache"] == 0
    line = cache.read_text().strip().split()
    assert len(line) == 4 and int(line[1]) == r["backend"] and int(line[2]) == r["ref_refresh"]
    r2 = Q.autotune(g, 0.8, cache_path=cache)
    assert r2["from_cache"] == 1 and r2["backend"] == r["backend"] and r2["ref_refresh"] == r["ref_refresh"]
    # the heavy-tailed graph has nnz(H) ~ 16 N: the CSR kernel wins
    assert r["backend"] == Q.QPR_BACKEND_SPARSE
    s = Q.Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, backend=r["backend"],
                            ref_refresh=r["ref_refresh"])
    assert s.backend == r["backend"]
