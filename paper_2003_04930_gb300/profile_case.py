"""Run a few RK4 steps of one workload, for profiler captures.

    python -m paper_2003_04930_gb300.profile_case --n 922 --omega 0.8 --backend sparse --steps 5 \
        [--precision mixed] [--sparse-form columns|persistent|gather|tiles] [--seed S] [--row-splits R]
        [--rkf45 ATTEMPTS]

Builds the heavy-tailed graph (seed 1 unless --seed), evolves rho0 = I/N by
`--steps` RK4 steps of dt = 0.01 through qpr_evolve (one CUDA graph launch
per 32 steps, or plain launches with --graph-steps 0), and prints the
per-kernel timing of qpr_profile_step (`--profile-steps` steps, each kernel
alone between CUDA events). With --rkf45 K it runs K attempts of qpr_rkf45
(fifth order) instead, for launch lists of the RKF45 kernels. Exit status 0
on success.
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

FORMS = {"auto": 0, "columns": 1, "tiles": 2, "persistent": 3, "gather": 5}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=922)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--omega", type=float, default=0.8)
    ap.add_argument("--backend", choices=["auto", "dense", "sparse"], default="sparse")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--graph-steps", type=int, default=0)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--sparse-form", choices=sorted(FORMS), default="auto")
    ap.add_argument("--row-splits", type=int, default=0)
    ap.add_argument("--rkf45", type=int, default=0,
                    help="instead of the RK4 profile: this many RKF45 attempts (fifth order, h0 = dt, Tol 1e-6)")
    a = ap.parse_args()
    import torch
    from paper_2003_04930_gb300 import Solver, graphs, qpr
    from paper_2003_04930_gb300.build import build_library
    build_library()
    be = {"auto": qpr.QPR_BACKEND_AUTO, "dense": qpr.QPR_BACKEND_DENSE, "sparse": qpr.QPR_BACKEND_SPARSE}
    g = graphs.heavy_tailed(a.n, a.seed)
    prec = {"fp64": qpr.QPR_FP64, "mixed": qpr.QPR_MIXED}[a.precision]
    s = Solver.from_edges(g, alpha=0.85, omega=a.omega, backend=be[a.backend], graph_steps=a.graph_steps,
                          precision=prec, sparse_form=FORMS[a.sparse_form], row_splits=a.row_splits)
    rho = torch.from_numpy(graphs.maximally_mixed(a.n)).cuda()
    if a.rkf45 > 0:
        st = s.rkf45(rho, tol=1e-14, max_steps=a.rkf45, h0=0.01, step_tol=1e-6, order=5, check=False)
        torch.cuda.synchronize()
        print(json.dumps({"rkf45_attempts": st["accepted"] + st["rejected"], "seconds": st["seconds"],
                          "kernel_launches": st["kernel_launches"], "sparse_form": s.sparse_form}))
        return 0
    s.evolve(rho, 0.01, a.steps)
    torch.cuda.synchronize()
    out = s.profile_step(rho, 0.01, a.profile_steps)
    out.update(sparse_form=s.sparse_form, sparse_plan=s.sparse_plan)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
