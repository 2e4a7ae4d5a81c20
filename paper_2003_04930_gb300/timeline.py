"""Where an RK4 step of the column-block mixed form goes, measured inside the
library's captured CUDA graphs (programmatic dependent launch on).

    python -m paper_2003_04930_gb300.timeline --n 922 --seed 1 --steps 256 [--sparse-form gather] [--json]

Builds and loads the diagnostic library libqpr_timeline.so (the column-block
kernels stamp the global timer when their first and last CTA enter and
leave, include/qpr_timeline.h), evolves rho0 = I/N on the heavy-tailed graph
for `--warm` steps, then times `--steps` steps and reports, per stage and as
medians over the steps (us):

  spmm      last SpMM-grid CTA out - last CTA out of the previous epilogue
  epilogue  last epilogue CTA out - last SpMM-grid CTA out
  staged    first / last product CTA with its column block in shared memory
            (whole-block form), from the previous epilogue's end
  rows_done first / last product CTA done with its rows, same origin
  early     first SpMM CTA in - previous epilogue's end (negative: started
            early under programmatic dependent launch)

and the step period (last stage-4 epilogue CTA out, step to step). These are
the critical path of the step: a profiler serialises the launches and shows
each kernel alone. Diagnostic only: the product library has no timeline.
"""
import argparse
import ctypes
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

KINDS, LAUNCHES, FIELDS = 8, 2048, 8


def _median(v):
    v = sorted(x for x in v if x == x)
    if not v:
        return float("nan")
    m = len(v) // 2
    return v[m] if len(v) % 2 else 0.5 * (v[m - 1] + v[m])


def _pct(v, p):
    v = sorted(x for x in v if x == x)
    return v[min(len(v) - 1, int(p / 100.0 * len(v)))] if v else float("nan")


def analyse(stamps, counts, steps):
    """Per-stage medians (us) of the step decomposition from the raw stamps
    (a nested list [kind][launch][field] of ints) of `steps` consecutive
    steps starting at launch 0."""
    unset = (1 << 64) - 1

    def t(k, i, f):
        v = stamps[k][i % LAUNCHES][f]
        return float("nan") if v in (unset, 0) else float(v)

    # launches 0 .. steps - 1 of every kind are the timed steps (a run that
    # stops mid-block launches the rest of the block's kernels, which return
    # at once: those come after)
    n = min(steps, LAUNCHES)
    per_stage = [dict(spmm=[], epilogue=[], early=[], staged_first=[], staged_last=[], rows_first=[], rows_last=[])
                 for _ in range(4)]
    period = []
    for i in range(1, n):
        prev = t(7, i - 1, 3)
        period.append((t(7, i, 3) - prev) / 1e3)
        for st in range(4):
            ks, ke = 2 * st, 2 * st + 1
            s_out, e_out = t(ks, i, 3), t(ke, i, 3)
            d = per_stage[st]
            d["spmm"].append((s_out - prev) / 1e3)
            d["epilogue"].append((e_out - s_out) / 1e3)
            d["early"].append((t(ks, i, 0) - prev) / 1e3)
            d["staged_first"].append((t(ks, i, 4) - prev) / 1e3)
            d["staged_last"].append((t(ks, i, 5) - prev) / 1e3)
            d["rows_first"].append((t(ks, i, 6) - prev) / 1e3)
            d["rows_last"].append((t(ks, i, 7) - prev) / 1e3)
            prev = e_out
    out = {"steps": n - 1, "step_period_us": _median(period), "step_period_p10_us": _pct(period, 10),
           "step_period_p90_us": _pct(period, 90), "stages": []}
    for st in range(4):
        out["stages"].append({k: _median(v) for k, v in per_stage[st].items()})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=922)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--omega", type=float, default=0.8)
    ap.add_argument("--steps", type=int, default=256)
    ap.add_argument("--warm", type=int, default=64)
    ap.add_argument("--sparse-form", choices=["auto", "columns", "gather"], default="auto")
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args()
    if a.steps >= LAUNCHES:
        raise SystemExit("--steps must be below %d" % LAUNCHES)
    from paper_2003_04930_gb300.build import build_library
    path = build_library(timeline=True)
    from paper_2003_04930_gb300 import qpr
    qpr.load_library(path)  # the first load of the process: the diagnostic library
    lib = ctypes.CDLL(path)
    lib.qpr_timeline_reset.restype = ctypes.c_int
    lib.qpr_timeline_read.restype = ctypes.c_int
    import torch
    from paper_2003_04930_gb300 import Solver, graphs
    form = {"auto": qpr.QPR_SPARSE_FORM_AUTO, "columns": qpr.QPR_SPARSE_FORM_COLUMNS,
            "gather": qpr.QPR_SPARSE_FORM_COLUMNS_GATHER}[a.sparse_form]
    g = graphs.heavy_tailed(a.n, a.seed)
    s = Solver.from_edges(g, alpha=0.85, omega=a.omega, precision=qpr.QPR_MIXED, backend=qpr.QPR_BACKEND_SPARSE,
                          sparse_form=form)
    if s.sparse_form not in (qpr.QPR_SPARSE_FORM_COLUMNS, qpr.QPR_SPARSE_FORM_COLUMNS_GATHER):
        raise SystemExit("the timeline covers the column-block forms only")
    rho = torch.from_numpy(graphs.maximally_mixed(a.n)).to("cuda")
    s.evolve(rho, 0.01, a.warm)
    torch.cuda.synchronize()
    if lib.qpr_timeline_reset() != 0:
        raise SystemExit("qpr_timeline_reset failed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.evolve(rho, 0.01, a.steps)
    e1.record()
    torch.cuda.synchronize()
    buf = (ctypes.c_ulonglong * (KINDS * LAUNCHES * FIELDS))()
    cnt = (ctypes.c_ulonglong * KINDS)()
    if lib.qpr_timeline_read(buf, cnt) != 0:
        raise SystemExit("qpr_timeline_read failed")
    flat = list(buf)
    stamps = [[flat[(k * LAUNCHES + i) * FIELDS:(k * LAUNCHES + i + 1) * FIELDS] for i in range(LAUNCHES)]
              for k in range(KINDS)]
    out = analyse(stamps, list(cnt), a.steps)
    out.update(n=a.n, seed=a.seed, omega=a.omega, sparse_form=s.sparse_form, sparse_plan=s.sparse_plan,
               evolve_ms_per_step=e0.elapsed_time(e1) / a.steps, launches=[int(c) for c in cnt])
    if a.json:
        print(json.dumps(out))
        return 0
    print("N=%d seed=%d omega=%.2f form=%d plan=%s" % (a.n, a.seed, a.omega, s.sparse_form, s.sparse_plan))
    print("evolve: %.2f us per step (events, refreshes included); step period median %.2f us (p10 %.2f, p90 %.2f)"
          % (1e3 * out["evolve_ms_per_step"], out["step_period_us"], out["step_period_p10_us"],
             out["step_period_p90_us"]))
    print("stage  spmm  epilogue  early  staged(first,last)  rows_done(first,last)   [us]")
    for st, d in enumerate(out["stages"]):
        print("%5d %5.2f %9.2f %6.2f   %6.2f %6.2f         %6.2f %6.2f" % (
            st + 1, d["spmm"], d["epilogue"], d["early"], d["staged_first"], d["staged_last"], d["rows_first"],
            d["rows_last"]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
