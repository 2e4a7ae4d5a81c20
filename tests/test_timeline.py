"""The diagnostic timeline build (include/qpr_timeline.h): its exports, the
product library's lack of them, the host-side decomposition of a step, and on
the GPU one short run whose parts add up to the step period."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

from paper_2003_04930_gb300 import timeline
from paper_2003_04930_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
UNSET = (1 << 64) - 1


def _empty():
    return [[[UNSET if f % 2 == 0 else 0 for f in range(timeline.FIELDS)] for _ in range(timeline.LAUNCHES)]
            for _ in range(timeline.KINDS)]


def test_exports_only_in_the_diagnostic_build():
    product = ctypes.CDLL(build_library())
    diag = ctypes.CDLL(build_library(timeline=True))
    for name in ("qpr_timeline_reset", "qpr_timeline_read"):
        assert hasattr(diag, name)
        assert not hasattr(product, name)


def test_decomposition_of_synthetic_steps():
    # every stage: the SpMM grid ends 9 us after the previous epilogue, the
    # epilogue 4 us after the SpMM grid (a 52 us step); the SpMM starts 1 us
    # early, its product CTAs are staged at 2 / 3 us and done at 8 / 9 us
    st = _empty()
    t = 1_000_000
    steps = 6
    for i in range(steps):
        for s in range(4):
            ks, ke = 2 * s, 2 * s + 1
            st[ks][i][0] = t - 1000
            st[ks][i][4], st[ks][i][5] = t + 2000, t + 3000
            st[ks][i][6], st[ks][i][7] = t + 8000, t + 9000
            st[ks][i][3] = t + 9000
            st[ke][i][3] = t + 13000
            t += 13000
    out = timeline.analyse(st, [0] * timeline.KINDS, steps)
    assert out["steps"] == steps - 1
    assert out["step_period_us"] == pytest.approx(52.0)
    for d in out["stages"]:
        assert d["spmm"] == pytest.approx(9.0) and d["epilogue"] == pytest.approx(4.0)
        assert d["early"] == pytest.approx(-1.0)
        assert (d["staged_first"], d["staged_last"]) == (pytest.approx(2.0), pytest.approx(3.0))
        assert (d["rows_first"], d["rows_last"]) == (pytest.approx(8.0), pytest.approx(9.0))


@pytest.mark.gpu
def test_timeline_run_adds_up():
    r = subprocess.run([sys.executable, "-m", "paper_2003_04930_gb300.timeline", "--n", "300", "--seed", "2",
                        "--steps", "64", "--warm", "8", "--json"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    parts = sum(d["spmm"] + d["epilogue"] for d in out["stages"])
    assert out["step_period_us"] > 0
    assert parts == pytest.approx(out["step_period_us"], rel=0.1)
    for d in out["stages"]:
        assert d["spmm"] > 0 and d["epilogue"] > 0
        assert d["staged_first"] <= d["staged_last"] <= d["rows_last"] <= d["spmm"] + 0.5
