"""qpr_profile_chain: the stage-2 SpMM grid and epilogue timed inside chains
of back-to-back launches with programmatic dependent launch, against the
same kernels launched alone (qpr_profile_step); the call leaves rho alone
and refuses forms it does not cover."""
import numpy as np
import pytest
import torch

from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n,seed,form", [(922, 1, Q.QPR_SPARSE_FORM_COLUMNS), (2048, 2, Q.QPR_SPARSE_FORM_COLUMNS_GATHER)])
def test_chain_times_are_kernel_times(n, seed, form):
    g = graphs.heavy_tailed(n, seed)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                          sparse_form=form)
    rho = torch.from_numpy(graphs.maximally_mixed(n)).to(DEV)
    s.evolve(rho, 0.01, 40)
    before = rho.clone()
    alone = s.profile_step(rho, 0.01, 4)
    chain = s.profile_chain(rho, 0.01, 20)
    assert torch.equal(rho, before)
    for k in ("product_ms", "epilogue_ms"):
        assert 0.0 < chain[k]
        # inside a chain the prologue overlaps the previous launch: not slower than alone (1 us slack)
        assert chain[k] <= alone[k] + 1e-3, (k, chain[k], alone[k])
    # the chain ran real stage work: the solve goes on from rho as before
    ref = before.clone()
    s.evolve(ref, 0.01, 8)
    s.evolve(rho, 0.01, 8)
    assert torch.equal(rho, ref)


def test_chain_refuses_other_forms_and_bad_arguments():
    g = graphs.heavy_tailed(200, 3)
    rho = torch.from_numpy(graphs.maximally_mixed(200)).to(DEV)
    for kw in (dict(), dict(precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE,
                            sparse_form=Q.QPR_SPARSE_FORM_TILES)):
        s = Solver.from_edges(g, alpha=0.85, omega=0.8, **kw)
        with pytest.raises(Q.QprError) as e:
            s.profile_chain(rho, 0.01, 4)
        assert e.value.status == Q.QPR_E_ARG
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
    for reps in (0, 5000):
        with pytest.raises(Q.QprError) as e:
            s.profile_chain(rho, 0.01, reps)
        assert e.value.status == Q.QPR_E_ARG


def test_log_line_on_stderr():
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import torch; from paper_2003_04930_gb300 import Solver, graphs; "
            "g = graphs.heavy_tailed(120, 4); s = Solver.from_edges(g, alpha=0.85, omega=0.8); "
            "r = torch.from_numpy(graphs.maximally_mixed(120)).to('cuda:0'); s.steady_state(r, 0.01, 1e-6, 100000)")
    env = dict(os.environ, QPR_LOG="1")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = [l for l in out.stderr.splitlines() if l.startswith("qpr_steady_state:")]
    assert len(line) == 1 and "N=120" in line[0] and "status=" in line[0]
