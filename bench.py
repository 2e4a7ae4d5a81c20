#!/usr/bin/env python
"""Benchmark: time-to-steady-state of the quantum PageRank RK4 solver.

Workload (the airline-sized case): heavy-tailed preferential-attachment
digraph, N = 922, seed 1 (power-law out-degrees, exponent 2.2, mean 8,
lognormal(0, 1) weights), alpha = 0.85, omega = 0.8, rho0 = I/N, classical
RK4 with dt = 0.01 until ||f(rho_n)||_F < 1e-8, complex128 state.

One benchmark step is one complete solve to the residual tolerance (every
RK4 step of it: stage operands, H rho, gain G p, fused epilogue, residual and
trace reductions, stop decision). `value` is seconds per solve (lower is
better); with N ranks each rank solves its own copy (replicas) and `value` is
the slowest rank's time divided by the solves of all ranks.

Besides the timed steps, rank 0 adds: the roofline of the dominant kernel
(each kernel timed alone by qpr_profile_step), the exact FP64 sparse form and
the plain dense FP64 (DMMA) form on the same problem, the learned warm start,
an end-to-end solve from pinned host memory, the same comparison at N = 4096
(`n4096`), one 512-graph batched solve (`batch512`) and the CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 C implementation) on a
bounded sample of RK4 steps of the same workload and scales it to one solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-steady-state (resid 1e-8) N=922/4096, warm+BF16 vs plain FP64; %TC peak"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0  # nominal dense FP64 / dense BF16 tensor rate of GB300
SMS = 152            # streaming multiprocessors of a GB300
SM_MAX_GHZ = 2.07    # maximum SM clock


def h_nonzeros(g):
    """Nonzeros of the off-diagonal H: ordered pairs (i, j), i != j, with a
    link i -> j or j -> i of nonzero weight."""
    import numpy as np
    src = np.asarray(g.src, dtype=np.int64)
    dst = np.asarray(g.dst, dtype=np.int64)
    w = np.ones(len(src)) if g.w is None else np.asarray(g.w, dtype=np.float64)
    keep = (src != dst) & (w != 0)
    a, b = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep])
    return 2 * int(np.unique(a * (int(g.n) + 1) + b).size)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=922)
    ap.add_argument("--omega", type=float, default=0.8)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--backend", choices=["auto", "dense", "sparse"], default="auto")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--ref-refresh", type=int, default=32)
    ap.add_argument("--no-fp64-sparse", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense-projection", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=0, help="oracle RK4 steps per sample (0: auto)")
    ap.add_argument("--workload", choices=["single", "batch"], default="single",
                    help="batch: qpr_batch_steady_state over --batch-count graphs (N ~ U[32,1024], "
                         "omega ~ U[0.1,0.95], seeds 1000+g)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-large", action="store_true", help="skip the N=4096 sub-object")
    ap.add_argument("--large-n", type=int, default=4096)
    ap.add_argument("--large-seed", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-graph batch sub-object")
    ap.add_argument("--no-omega-sweep", action="store_true", help="skip the omega in {0.2, 0.5, 1.0} sub-object")
    ap.add_argument("--cpu-omega-sweep", action="store_true",
                    help="add the CPU oracle's whole solves to the omega sweep (minutes of host time)")
    ap.add_argument("--cpu-full-max-s", type=float, default=90.0,
                    help="run the oracle solve to completion when its estimate is below this many seconds")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def workload_config(a):
    return {"workload": f"heavy-tailed PA digraph N={a.n} seed={a.seed} (gamma 2.2, mean out-degree 8, "
                        f"lognormal(0,1) weights), alpha=0.85, omega={a.omega}, rho0=I/N, RK4 dt={a.dt}, "
                        f"until ||L(rho)||_F<{a.tol}, complex128",
            "n": a.n, "omega": a.omega, "dt": a.dt, "tol": a.tol, "alpha": 0.85,
            "l2": "flushed between timed solves (256 MiB write); the 4 FP64 state buffers "
                  f"({4 * 16 * a.n * a.n / 2**20:.0f} MiB at N={a.n}) stay L2-resident within a solve"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


# ---------------------------------------------------------------- oracle
def cpu_baseline(a, steps_to_converge: int, sample_steps: int = 0):
    """The CPU oracle on the same workload, on all host cores: the whole
    solve to the residual tolerance when its estimate (a short probe) is below
    --cpu-full-max-s, else a bounded sample of RK4 steps scaled to the solve's
    step count. Also a single-thread sample (seconds per RK4 step)."""
    from oracle import Oracle
    from oracle.cpu import max_threads, set_threads
    from paper_2003_04930_gb300 import graphs

    g = graphs.heavy_tailed(a.n, a.seed)
    o = Oracle.from_edges(g, alpha=0.85, omega=a.omega)
    rho0 = graphs.maximally_mixed(a.n)
    cores = max_threads()
    probe = 4
    t = time.perf_counter()
    o.evolve(rho0, a.dt, probe)
    per = (time.perf_counter() - t) / probe
    out = {"unit": "s", "cores": cores, "kind": "oracle"}
    if not sample_steps and per * steps_to_converge <= a.cpu_full_max_s:
        t = time.perf_counter()
        _, steps, resid, _ = o.steady_state(rho0, a.dt, a.tol, a.max_steps)
        el = time.perf_counter() - t
        out.update(value=el, sample=f"the whole solve to ||f||_F < {a.tol}: {steps} RK4 steps, final residual "
                                    f"{resid:.3e}, run to completion on {cores} threads",
                   steps=steps, seconds_per_rk4_step=el / max(steps, 1), projected=False)
    else:
        r = sample_steps or max(2, min(steps_to_converge, int(15.0 / max(per, 1e-6))))
        t = time.perf_counter()
        o.evolve(rho0, a.dt, r)
        el = time.perf_counter() - t
        out.update(value=el / r * steps_to_converge, projected=True,
                   sample=f"{r} RK4 steps of the same workload timed ({el:.1f} s), scaled by the "
                          f"{steps_to_converge} steps the solve takes", seconds_per_rk4_step=el / r)
    # one thread: a bounded sample of steps (about 5 s), seconds per step
    set_threads(1)
    try:
        r1 = max(2, min(200, int(5.0 / max(per * cores, 1e-6))))
        t = time.perf_counter()
        o.evolve(rho0, a.dt, r1)
        el1 = time.perf_counter() - t
    finally:
        set_threads(cores)
    out["single_thread"] = {"seconds_per_rk4_step": el1 / r1, "sample_steps": r1,
                            "projected_solve_s": el1 / r1 * steps_to_converge}
    return out


def oracle_steps_to_converge(a):
    """Step count of the oracle solve from the committed oracle output."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_steady_n922.json")
    if a.n == 922 and a.seed == 1 and abs(a.dt - 0.01) < 1e-15 and a.tol == 1e-8 and os.path.exists(p):
        d = json.load(open(p))
        if str(a.omega) in d:
            return int(d[str(a.omega)]["steps"])
    return None


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps = oracle_steps_to_converge(a)
    if steps is None:
        print(json.dumps({"impl": "reference", "unavailable": "no oracle step count stored for this workload"}))
        return 0
    from oracle import Oracle
    from oracle.cpu import max_threads
    from paper_2003_04930_gb300 import graphs
    g = graphs.heavy_tailed(a.n, a.seed)
    o = Oracle.from_edges(g, alpha=0.85, omega=a.omega)
    rho = graphs.maximally_mixed(a.n)
    sample = a.cpu_sample_steps or 100
    vals = []
    for k in range(a.warmup + a.steps):
        t = time.perf_counter()
        rho = o.evolve(rho, a.dt, sample)
        el = time.perf_counter() - t
        if k >= a.warmup:
            vals.append(el / sample * steps)
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference", "config": workload_config(a),
            "cpu_baseline": {"value": v, "unit": "s", "cores": max_threads(), "kind": "oracle",
                             "sample": f"each step: {sample} oracle RK4 steps, scaled by the {steps} "
                                       f"steps of one solve"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours
def replica_time(local_total, steps, dist=None, device=None):
    """Replicas (one independent solve stream per rank): the slowest rank's
    timed total, max over ranks, and the time per solve over the solves of
    all ranks. Returns (seconds per solve, max total)."""
    import torch

    world = 1
    total = float(local_total)
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([total], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total / (steps * world), total


def run_ours(a):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2003_04930_gb300 import Solver, graphs, qpr
    from paper_2003_04930_gb300.build import build_library
    build_library()

    backend = {"auto": qpr.QPR_BACKEND_AUTO, "dense": qpr.QPR_BACKEND_DENSE,
               "sparse": qpr.QPR_BACKEND_SPARSE}[a.backend]
    prec = {"fp64": qpr.QPR_FP64, "mixed": qpr.QPR_MIXED}[a.precision]
    g = graphs.heavy_tailed(a.n, a.seed)
    s = Solver.from_edges(g, alpha=0.85, omega=a.omega, backend=backend, device=local, precision=prec,
                          ref_refresh=a.ref_refresh)
    rho0 = torch.from_numpy(graphs.maximally_mixed(a.n)).to(dev)
    rho = torch.empty_like(rho0)
    flush = torch.empty(64 * 2**20, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def solve():
        rho.copy_(rho0)
        return s.steady_state(rho, a.dt, a.tol, a.max_steps)

    for _ in range(a.warmup):
        solve()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    times, stats = [], []
    for _ in range(a.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = solve()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        stats.append(st)
    barrier()
    clocks = sampler.stop()
    value, total = replica_time(sum(times), a.steps, dist, dev)
    steps_conv = stats[-1]["steps"]
    n = a.n
    rho_solved = rho.clone()  # this form's steady state, compared with the FP64 sparse form's below

    # per-kernel durations on the solver's stream, same workload and state: each kernel alone between events
    peaks, peak_src = load_peaks()
    prof = s.profile_step(rho, a.dt, 20)
    chain = s.profile_chain(rho, a.dt, CHAIN_REPS) if column_form(s, prec) else None
    roof = roofline(s, g, a.n, prof, peaks, peak_src, prec, chain)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == qpr.QPR_FP64 else "f32+f64", "data": "synthetic",
            "config": dict(workload_config(a), form=form_name(s, prec), ref_refresh=a.ref_refresh,
                           sparse_plan=s.sparse_plan, parallelism=f"replicas{world}"),
            "rk4_steps_to_converge": steps_conv, "rk4_steps_per_s": steps_conv / (total / a.steps),
            "residual": stats[-1]["residual"], "roofline": roof, "profile_ms": prof, "profile_chain_ms": chain,
            "clocks": clocks,
            "gpu_launches": int(sum(st["kernel_launches"] for st in stats))}

    # the paper's own integrator: adaptive RKF45 (Supplementary Note 2) on the same problem and stop rule
    if prec == qpr.QPR_MIXED and s.sparse_form in (qpr.QPR_SPARSE_FORM_COLUMNS, qpr.QPR_SPARSE_FORM_COLUMNS_GATHER):
        line["rkf45"] = rkf45_solve(s, a, rho0, rho_solved, flush, max(1, a.steps), value, steps_conv)

    # the main text's comparison of the quantum and the classical ranking: hub classes (c = 10) of the
    # steady-state populations and of the classical PageRank vector, both on the GPU
    line["hubs"] = hub_report(s, rho_solved)

    # the plain dense FP64 (DMMA) form on the same problem: s/step x steps
    if not a.no_dense_projection and s.backend != qpr.QPR_BACKEND_DENSE:
        line["plain_fp64_dense"] = dense_projection(g, a.omega, local, rho, a.dt, steps_conv, peaks, peak_src)

    # the exact FP64 sparse form on the same problem, one solve
    if not a.no_fp64_sparse and (prec != qpr.QPR_FP64 or s.backend != qpr.QPR_BACKEND_SPARSE):
        line["fp64_sparse"] = fp64_sparse_solve(g, a, local, rho0, rho_solved, flush, warm=True)

    # the learned warm start (network trained by train_warmstart, weights in the package): inference plus the
    # solve from rho0 = diag(p_hat), timed like the cold solve
    if not a.no_warm_start and prec == qpr.QPR_MIXED:
        ws = warm_solve(s, g, a.omega, a, local, rho, flush, max(1, a.steps))
        if ws is not None:
            ws.update(cold_steps=steps_conv, cold_value=value)
            line["warm_start"] = ws

    # end to end through the C ABI with host buffers (pinned), copies inside
    host = torch.empty((n, n), dtype=torch.complex128, pin_memory=True)
    host0 = rho0.cpu()
    e2e = []
    for _ in range(max(1, a.steps)):
        host.copy_(host0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.steady_state(host, a.dt, a.tol, a.max_steps)
        e2e.append(time.perf_counter() - t)
    line["e2e"] = {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": 16 * n * n,
                   "d2h_bytes_per_step": 16 * n * n}
    s.close()

    # the other size the metric names, the batched form and the omega sweep: one-GPU facts, measured in the
    # N = 1 run only (with N ranks every GPU would wait on rank 0 meanwhile)
    if not a.no_large and rank == 0 and world == 1:
        line["n4096"] = large_case(a, local, peaks, peak_src, flush)
    if not a.no_batch and rank == 0 and world == 1:
        line["batch512"] = batch_case(a, local)
    if not a.no_omega_sweep and rank == 0 and world == 1 and a.n == 922:
        line["omega_sweep"] = omega_sweep(a, local, flush, cpu=a.cpu_omega_sweep and world == 1)

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, steps_conv, a.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def rkf45_solve(s, a, rho0, rho_ref, flush, reps, rk4_value, rk4_steps, step_tol=1e-6, order=5):
    """qpr_rkf45 to the same residual tolerance from the same start (h0 =
    dt, Tol = 1e-6, h_max = the RK4 stability estimate), propagating the
    fifth-order solution z of Eq. S12 (the note's alternative; the
    fourth-order y stalls where the coherences are weakly damped), one
    untimed solve then `reps` timed with CUDA events; the difference of its
    steady state from the fixed-step RK4 one (both stop at ||f||_F < tol, so
    they differ by up to about tol over the spectral gap). Also the step
    counts of one fourth-order solve, for comparison."""
    import torch
    kw = dict(tol=a.tol, max_steps=min(a.max_steps, 100000), h0=a.dt, step_tol=step_tol)
    rho = torch.empty_like(rho0)
    rho.copy_(rho0)
    s.rkf45(rho, order=order, **kw)
    ts, st = [], None
    for _ in range(reps):
        rho.copy_(rho0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = s.rkf45(rho, order=order, **kw)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.mean(ts)
    p, pr = torch.diagonal(rho).real, torch.diagonal(rho_ref).real
    out = {"time_to_steady_state_s": t, "order": order, "accepted_steps": st["accepted"],
           "rejected": st["rejected"], "t": st["t"], "h_final": st["h_next"], "h_max": s.max_stable_dt,
           "step_tol": step_tol, "residual": st["residual"], "gpu_launches": st["kernel_launches"],
           "rk4_steps": rk4_steps, "rk4_time_s": rk4_value, "speedup_vs_rk4": rk4_value / t,
           "max_dp_rel_vs_rk4": float((p - pr).abs().max() / pr.abs().max()),
           "form": "mixed column-block form, six powers of h L per attempt, controller on the device"}
    rho.copy_(rho0)
    t4 = time.perf_counter()
    kw4 = dict(kw, max_steps=4 * st["accepted"] + 100)  # bounded: the fourth-order solution can stall
    st4 = s.rkf45(rho, order=4, check=False, **kw4)
    torch.cuda.synchronize()
    out["order4"] = {"status": st4["status"], "converged": st4["converged"], "accepted_steps": st4["accepted"],
                     "rejected": st4["rejected"], "t": st4["t"], "residual": st4["residual"],
                     "max_steps": kw4["max_steps"], "wall_s": time.perf_counter() - t4}
    return out


def hub_report(s, rho_ss, c=10.0, top=10):
    """QPR against classical PageRank on the solved graph: hub counts (main
    p > c/N, secondary 1/N < p <= c/N) of both vectors, the overlap of their
    hub sets and of their top-`top` nodes (qpr_populations, qpr_pagerank,
    qpr_hub_classes)."""
    import numpy as np
    p, rank = s.populations(rho_ss, with_rank=True)
    t = time.perf_counter()
    pi = s.pagerank(tol=1e-14)
    t_pr = time.perf_counter() - t
    cq, nq = s.hub_classes(p, c)
    cp, npr = s.hub_classes(pi, c)
    rank_pr = np.argsort(-pi, kind="stable")
    return {"c": c, "qpr_counts": {"main": int(nq[2]), "secondary": int(nq[1])},
            "pagerank_counts": {"main": int(npr[2]), "secondary": int(npr[1])},
            "main_hubs_in_both": int(np.sum((cq == 2) & (cp == 2))),
            "hubs_in_both": int(np.sum((cq >= 1) & (cp >= 1))),
            f"top{top}_overlap": len(set(rank[:top].tolist()) & set(rank_pr[:top].tolist())),
            "qpr_top": rank[:top].tolist(), "pagerank_top": rank_pr[:top].tolist(),
            "pagerank_iters": s.last_pagerank_iters, "pagerank_s": t_pr}


def form_name(s, prec):
    from paper_2003_04930_gb300 import qpr
    form = {(qpr.QPR_FP64, 1): "fp64 dense DMMA", (qpr.QPR_FP64, 2): "fp64 sparse CSR",
            (qpr.QPR_MIXED, 1): "mixed: split-BF16 tcgen05 GEMM deltas (FP32 accumulate) + fp64 "
                                "reference/accumulation/residual",
            (qpr.QPR_MIXED, 2): "mixed: fp32 sparse CSR deltas (tile pairs) + float-float delta "
                                "accumulation + fp64 reference/residual"}[(prec, s.backend)]
    if s.sparse_form in (qpr.QPR_SPARSE_FORM_COLUMNS, qpr.QPR_SPARSE_FORM_COLUMNS_PERSISTENT):
        form = ("mixed: fp32 column-block SpMM from TMA-staged shared memory + tile-pair epilogue, "
                "float-float delta accumulation, fp64 reference/residual")
    elif s.sparse_form == qpr.QPR_SPARSE_FORM_COLUMNS_GATHER:
        form = ("mixed: fp32 column-block SpMM gathering row segments through L1/L2 + tile-pair epilogue, "
                "float-float delta accumulation, fp64 reference/residual")
    return form


# DRAM bytes per launch of the current kernels from one ncu capture each
# (`dram__bytes_read.sum + dram__bytes_write.sum` of the stage-1 launch, and
# of the stage-2 epilogue,
# profiles/traffic_cols_n922_n4096.md), keyed by (kernel, N); a kernel
# changed since its capture has no entry.
NCU_TRAFFIC = {("cols_spmm_kernel", 922): 7127808, ("cols_epi_kernel", 922): 14042880,
               ("cols_epi_kernel_stage2", 922): 17606144,
               ("cols_gather_kernel", 4096): 135363584 + 100583424, ("cols_epi_kernel", 4096): 269675520 + 101277440,
               ("cols_epi_kernel_stage2", 4096): 337357312 + 104324864}


def column_form(s, prec):
    """True when the solver runs a column-block form (qpr_profile_chain applies)."""
    from paper_2003_04930_gb300 import qpr
    return (prec == qpr.QPR_MIXED and s.backend == qpr.QPR_BACKEND_SPARSE and
            s.sparse_form != qpr.QPR_SPARSE_FORM_TILES)


CHAIN_REPS = 20
CHAIN_SOURCE = (f"qpr_profile_chain: {CHAIN_REPS} launches of the kernel back to back with programmatic dependent "
                "launch (as in the solve's graphs), CUDA events around the chain on the launching stream")
ALONE_SOURCE = "qpr_profile_step: the kernel alone on the stream between two CUDA events"


def roofline(s, g, n, prof, peaks, peak_src, prec, chain=None):
    """Roofline of the dominant kernel of the form in use, from the kernel's
    duration inside a chain of launches (qpr_profile_chain, column-block
    forms: `chain`) or launched alone (qpr_profile_step: `prof`)."""
    from paper_2003_04930_gb300 import qpr
    hbm = peaks["hbm_gbs"]

    def hbm_entry(kernel, alg, ms, extra=None, source=ALONE_SOURCE, key=None):
        ach = alg / (ms * 1e-3) / 1e9
        d = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
             "traffic": NCU_TRAFFIC.get(key or (kernel, n)), "kernel": kernel, "alg_bytes_per_launch": alg,
             "launch_ms": ms, "peak_source": f"hbm_gbs of {peak_src}", "launch_ms_source": source}
        if extra:
            d.update(extra)
        return d

    if s.backend == qpr.QPR_BACKEND_DENSE and prec == qpr.QPR_MIXED:
        # split-BF16 GEMM: 6 BF16 products of H (np x np) with [Re | Im] delta (np x 2 np), on the padded np
        npad = ((n + 127) // 128) * 128
        flops = 6 * 2.0 * npad * (2 * npad) * npad
        ach = flops / (prof["product_ms"] * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "frac": ach / peaks["bf16_tflops"], "traffic": None, "kernel": "stage_mixed_tc_kernel (tcgen05)",
                "alg_flops_per_launch": flops, "launch_ms": prof["product_ms"],
                "peak_source": f"bf16_tflops of {peak_src}"}
    if s.backend == qpr.QPR_BACKEND_SPARSE and prec == qpr.QPR_MIXED and s.sparse_form != qpr.QPR_SPARSE_FORM_TILES:
        gather = s.sparse_form == qpr.QPR_SPARSE_FORM_COLUMNS_GATHER
        npad = ((n + 31) // 32) * 32
        nnz = h_nonzeros(g)
        # SpMM: one read of the stage input and one write of X (two FP32 planes each, 8 np^2 bytes), and the
        # CSR entries of H once (8 bytes per nonzero, column index and FP32 value)
        alg = 16 * npad * npad + 8 * nnz
        kernel = "cols_gather_kernel" if gather else "cols_spmm_kernel"
        # epilogue (nested RK4 form): FP32 plane pairs (8 bytes per element) read or written per stage:
        # stage 1 X, D, F32, the next input (32); stages 2-3 X, the input, F32, D, the next input (40);
        # stage 4 X, the input, D, Dlo, Ghi, Glo, D and Dlo written (64): mean (32 + 40 + 40 + 64) / 4 = 44
        epi_alg = 44 * n * n
        rows_read = nnz * npad * 8  # each nonzero's row of the stage input, per column block (L1/L2 or smem)
        if chain is not None:
            # the chains repeat the stage-2 kernels: its epilogue moves 40 bytes per element
            spmm_ms, src = chain["product_ms"], CHAIN_SOURCE
            epi = hbm_entry("cols_epi_kernel", 40 * n * n, chain["epilogue_ms"], source=CHAIN_SOURCE,
                            key=("cols_epi_kernel_stage2", n),
                            extra={"stage": 2, "launch_ms_alone_mean_of_4_stages": prof["epilogue_ms"]})
        else:
            spmm_ms, src = prof["product_ms"], ALONE_SOURCE
            epi = hbm_entry("cols_epi_kernel", epi_alg, prof["epilogue_ms"])
        extra = {"gathered_bytes_per_launch": rows_read,
                 "gathered_gbs": rows_read / (spmm_ms * 1e-3) / 1e9,
                 "flops_per_launch": 4.0 * nnz * npad,
                 "launch_ms_alone": prof["product_ms"],
                 "epilogue": epi,
                 "gain": "formed by the SpMM grid's leading CTAs (cta_gain), inside launch_ms",
                 "note": "alg bytes are the DRAM floor (stage input and X once, the CSR entries once); at "
                         "N <= 1400 the state is L2-resident, so a fraction of the HBM peak is a lower bound "
                         "on what the kernel moves through the memory system"}
        return hbm_entry(kernel, alg, spmm_ms, extra, source=src)
    if s.backend == qpr.QPR_BACKEND_SPARSE:
        if prec == qpr.QPR_MIXED:
            alg, kname = 52 * n * n, "stage_mixed_sparse_kernel"
        else:
            alg, kname = 4 * 16 * n * n, "stage_sparse_kernel"
        return hbm_entry(kname, alg, prof["product_ms"])
    flops = 4.0 * n ** 3
    fp64_peak = peaks["bf16_tflops"] * NOMINAL_FP64_OVER_BF16
    ach = flops / (prof["product_ms"] * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": ach / fp64_peak, "traffic": None, "kernel": "stage_fp64_kernel (DMMA)",
            "alg_flops_per_launch": flops, "launch_ms": prof["product_ms"],
            "peak_source": f"bf16_tflops of {peak_src} x nominal FP64/BF16 ratio 1.25/2250"}


def dense_projection(g, omega, local, rho, dt, steps_conv, peaks, peak_src, prof_steps=3):
    """The plain dense FP64 (DMMA) form on the same problem: its step time
    from qpr_profile_step times the step count of the solve (projected)."""
    from paper_2003_04930_gb300 import Solver, qpr
    sd = Solver.from_edges(g, alpha=0.85, omega=omega, backend=qpr.QPR_BACKEND_DENSE, device=local)
    pd = sd.profile_step(rho, dt, prof_steps)
    sd.close()
    flops = 4.0 * g.n ** 3
    fp64_peak = peaks["bf16_tflops"] * NOMINAL_FP64_OVER_BF16
    return {"ms_per_rk4_step": pd["step_ms"], "projected_time_to_steady_state_s": pd["step_ms"] * 1e-3 * steps_conv,
            "projected": True, "stage_tflops": flops / (pd["product_ms"] * 1e-3) / 1e12,
            "frac_of_fp64_peak": flops / (pd["product_ms"] * 1e-3) / 1e12 / fp64_peak,
            "fp64_peak_tflops": fp64_peak, "peak_source": f"bf16_tflops of {peak_src} x 1.25/2250"}


def tc_bf16_stage(g, omega, local, rho, dt, steps_conv, peaks, peak_src, prof_steps=2):
    """The dense split-BF16 tcgen05 form (the stage as one tensor-core GEMM
    of H against the split delta planes) on the same problem: its stage GEMM's rate against the measured
    BF16 peak (qpr_profile_step), and its step time times the step count of
    the solve (projected; the sparse forms are faster on these graphs)."""
    from paper_2003_04930_gb300 import Solver, qpr
    st = Solver.from_edges(g, alpha=0.85, omega=omega, backend=qpr.QPR_BACKEND_DENSE, precision=qpr.QPR_MIXED,
                           device=local)
    pd = st.profile_step(rho, dt, prof_steps)
    roof = roofline(st, g, g.n, pd, peaks, peak_src, qpr.QPR_MIXED)
    st.close()
    return {"kernel": roof["kernel"], "stage_tflops": roof["achieved"], "frac_of_bf16_peak": roof["frac"],
            "bf16_peak_tflops": roof["peak"], "peak_source": roof["peak_source"], "launch_ms": pd["product_ms"],
            "ms_per_rk4_step": pd["step_ms"], "projected_time_to_steady_state_s": pd["step_ms"] * 1e-3 * steps_conv,
            "projected": True}


def timed_solve(s, rho, rho0, a, flush):
    import torch
    rho.copy_(rho0)
    flush.fill_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    st = s.steady_state(rho, a.dt, a.tol, a.max_steps)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, st


def fp64_sparse_solve(g, a, local, rho0, rho_solved, flush, warm):
    """One solve of the exact FP64 sparse form (after one untimed solve when
    `warm`), and the error of `rho_solved` against it: the precision form's
    stated bounds are max|dp| <= 1e-7 max p and ||drho||_F <= 1e-6."""
    import torch
    from paper_2003_04930_gb300 import Solver, qpr
    sf = Solver.from_edges(g, alpha=0.85, omega=a.omega, backend=qpr.QPR_BACKEND_SPARSE, device=local)
    rho = torch.empty_like(rho0)
    if warm:
        rho.copy_(rho0)
        sf.steady_state(rho, a.dt, a.tol, a.max_steps)
    t, stf = timed_solve(sf, rho, rho0, a, flush)
    sf.close()
    p_ours = torch.diagonal(rho_solved).real
    p_fp64 = torch.diagonal(rho).real
    return {"time_to_steady_state_s": t, "steps": stf["steps"],
            "max_dp_rel": float((p_ours - p_fp64).abs().max() / p_fp64.abs().max()),
            "fro_drho": float(torch.linalg.norm(rho_solved - rho))}


def warm_solve(s, g, omega, a, local, rho, flush, reps):
    """GNN inference (qpr_gnn_predict) + rho0 = diag(p_hat) upload + solve,
    wall-clocked `reps` times after one untimed run; None when the network is
    absent or omega is below the warm-start threshold."""
    import torch
    from paper_2003_04930_gb300 import warmstart
    net = warmstart.load_network(device=local)
    if net is None or omega < warmstart.WARM_OMEGA_MIN:
        return None

    def once():
        p_hat = net.predict(g, omega)
        rho.copy_(torch.from_numpy(warmstart.warm_rho(p_hat)))
        return s.steady_state(rho, a.dt, a.tol, a.max_steps)
    once()
    wt, wst = [], None
    for _ in range(reps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        wst = once()
        torch.cuda.synchronize()
        wt.append(time.perf_counter() - t)
    net.close()
    return {"value": statistics.mean(wt), "unit": "s", "steps": wst["steps"],
            "timed": "GNN inference (qpr_gnn_predict) + rho0 = diag(p_hat) upload + solve",
            "network": "4-layer message passing, width 64, BF16 weights, trained on 256 solver-generated "
                       "steady states (N in [64, 1024])"}


SWEEP_OMEGAS = (0.2, 0.5, 1.0)


def omega_sweep(a, local, flush, cpu=False):
    """The headline graph at the other mixing values of the plain-FP64
    configuration (omega in {0.2, 0.5, 1.0}; 0.8 is the headline): per omega
    the mixed solve and the FP64 sparse solve (one untimed, one timed each),
    their steady states against each other, and RKF45 (fifth order, bounded);
    with `cpu`, the CPU oracle's whole solve on all host cores too."""
    import torch
    from paper_2003_04930_gb300 import Solver, graphs, qpr
    g = graphs.heavy_tailed(a.n, a.seed)
    dev = torch.device("cuda", local)
    rho0 = torch.from_numpy(graphs.maximally_mixed(a.n)).to(dev)
    out = {}
    for om in SWEEP_OMEGAS:
        sa = argparse.Namespace(**vars(a))
        sa.omega = om
        s = Solver.from_edges(g, alpha=0.85, omega=om, precision=qpr.QPR_MIXED, device=local,
                              ref_refresh=a.ref_refresh)
        rho = torch.empty_like(rho0)
        rho.copy_(rho0)
        s.steady_state(rho, a.dt, a.tol, a.max_steps)
        t_mixed, st = timed_solve(s, rho, rho0, sa, flush)
        rho_mixed = rho.clone()
        d = {"mixed": {"time_to_steady_state_s": t_mixed, "steps": st["steps"], "residual": st["residual"]}}
        rk = torch.empty_like(rho0)
        rk.copy_(rho0)
        # bounded by the RK4 step count: where the fifth-order solution stalls it is no alternative
        kmax = int(st["steps"])
        r = s.rkf45(rk, tol=a.tol, max_steps=kmax, h0=a.dt, step_tol=1e-6, order=5, check=False)
        rk.copy_(rho0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = s.rkf45(rk, tol=a.tol, max_steps=kmax, h0=a.dt, step_tol=1e-6, order=5, check=False)
        e1.record()
        e1.synchronize()
        d["rkf45"] = {"converged": r["converged"], "accepted_steps": r["accepted"], "rejected": r["rejected"],
                      "time_s": e0.elapsed_time(e1) / 1e3, "residual": r["residual"]}
        s.close()
        d["fp64_sparse"] = fp64_sparse_solve(g, sa, local, rho0, rho_mixed, flush, warm=True)
        d["speedup_vs_fp64_sparse"] = d["fp64_sparse"]["time_to_steady_state_s"] / t_mixed
        if cpu:
            from oracle import Oracle
            from oracle.cpu import max_threads
            o = Oracle.from_edges(g, alpha=0.85, omega=om)
            t = time.perf_counter()
            _, steps, resid, _ = o.steady_state(graphs.maximally_mixed(a.n), a.dt, a.tol, a.max_steps)
            d["cpu_oracle"] = {"time_to_steady_state_s": time.perf_counter() - t, "steps": steps,
                               "residual": resid, "cores": max_threads()}
        out[f"omega={om}"] = d
    return out


def tuned_solve(g, a, local, rho0, rho_solved, flush, t_fixed):
    """The autotuner's choice (qpr_autotune: backend, stage form, row splits,
    then the reference-refresh block, timed on the device; no cache file),
    one untimed and one timed solve of it, and its steady state against the
    fixed rule's."""
    import torch
    from paper_2003_04930_gb300 import Solver, qpr
    t0 = time.perf_counter()
    r = qpr.autotune(g, a.omega, dt=a.dt, precision=qpr.QPR_MIXED, device=local)
    tune_s = time.perf_counter() - t0
    st = Solver.from_edges(g, alpha=0.85, omega=a.omega, precision=qpr.QPR_MIXED, device=local,
                           **qpr.tuned_options(r))
    rho = torch.empty_like(rho0)
    rho.copy_(rho0)
    st.steady_state(rho, a.dt, a.tol, a.max_steps)
    t, stt = timed_solve(st, rho, rho0, a, flush)
    p, pr = st.populations(rho), st.populations(rho_solved)
    out = {"choice": {k: r[k] for k in ("backend", "sparse_form", "row_splits", "ref_refresh")},
           "sparse_plan": st.sparse_plan, "tune_s": tune_s, "tuner_ms_per_step": r["ms_per_step"],
           "time_to_steady_state_s": t, "steps": stt["steps"], "fixed_rule_s": t_fixed,
           "speedup_vs_fixed_rule": t_fixed / t,
           "max_dp_rel_vs_fixed_rule": float(abs(p - pr).max() / abs(pr).max())}
    st.close()
    return out


def large_case(a, local, peaks, peak_src, flush):
    """The metric's second size: the same generator at N = 4096 (seed 3),
    omega = 0.8. Mixed cold and warm-started solves (one timed each after one
    untimed), one FP64 sparse solve (the exact form, also the reference of
    the error), the plain dense FP64 DMMA form projected from one profiled
    step, and the roofline of the gather SpMM and the epilogue."""
    import torch
    from paper_2003_04930_gb300 import Solver, graphs, qpr
    n = a.large_n
    la = argparse.Namespace(**vars(a))
    la.n, la.seed = n, a.large_seed
    g = graphs.heavy_tailed(n, la.seed)
    dev = torch.device("cuda", local)
    s = Solver.from_edges(g, alpha=0.85, omega=la.omega, precision=qpr.QPR_MIXED, device=local,
                          ref_refresh=la.ref_refresh)
    rho0 = torch.from_numpy(graphs.maximally_mixed(n)).to(dev)
    rho = torch.empty_like(rho0)
    rho.copy_(rho0)
    s.steady_state(rho, la.dt, la.tol, la.max_steps)
    t_cold, st = timed_solve(s, rho, rho0, la, flush)
    rho_solved = rho.clone()
    out = {"workload": f"heavy-tailed PA digraph N={n} seed={la.seed}, alpha=0.85, omega={la.omega}, rho0=I/N, "
                       f"RK4 dt={la.dt}, until ||L(rho)||_F<{la.tol}",
           "form": form_name(s, qpr.QPR_MIXED), "sparse_plan": s.sparse_plan,
           "cold": {"time_to_steady_state_s": t_cold, "steps": st["steps"], "residual": st["residual"],
                    "gpu_launches": st["kernel_launches"]}}
    prof = s.profile_step(rho_solved, la.dt, 4)
    out["profile_ms"] = prof
    chain = s.profile_chain(rho_solved, la.dt, CHAIN_REPS) if column_form(s, qpr.QPR_MIXED) else None
    out["profile_chain_ms"] = chain
    out["roofline"] = roofline(s, g, n, prof, peaks, peak_src, qpr.QPR_MIXED, chain)
    ws = warm_solve(s, g, la.omega, la, local, rho, flush, 1)
    if ws is not None:
        out["warm_start"] = ws
    out["rkf45"] = rkf45_solve(s, la, rho0, rho_solved, flush, 1, t_cold, st["steps"])
    out["autotuned"] = tuned_solve(g, la, local, rho0, rho_solved, flush, t_cold)
    s.close()
    out["fp64_sparse"] = fp64_sparse_solve(g, la, local, rho0, rho_solved, flush, warm=False)
    out["plain_fp64_dense"] = dense_projection(g, la.omega, local, rho_solved, la.dt, st["steps"], peaks, peak_src,
                                               prof_steps=1)
    out["tc_bf16"] = tc_bf16_stage(g, la.omega, local, rho_solved, la.dt, st["steps"], peaks, peak_src)
    best = min(t_cold, ws["value"]) if ws is not None else t_cold
    out["speedup_vs_fp64_sparse"] = out["fp64_sparse"]["time_to_steady_state_s"] / best
    out["speedup_vs_plain_fp64_dense_projected"] = out["plain_fp64_dense"]["projected_time_to_steady_state_s"] / best
    return out


def batch_case(a, local):
    """The batched form: one qpr_batch_steady_state call over 512 graphs
    (N ~ U[32,1024], omega ~ U[0.1,0.95], seeds 1000+g), timed once (the
    call assembles, uploads and plans every problem itself, so there is no
    state for a warm-up call to leave behind)."""
    import numpy as np
    import torch
    from paper_2003_04930_gb300 import graphs, qpr
    specs = graphs.batch_specs(a.batch_count)
    gs = [graphs.heavy_tailed(n, seed) for n, om, seed in specs]
    dev = torch.device("cuda", local)
    rho0 = [torch.from_numpy(graphs.maximally_mixed(g.n)).to(dev) for g in gs]
    rho = [r.clone() for r in rho0]
    probs = [(g, om, r) for g, (n, om, seed), r in zip(gs, specs, rho)]

    def solve():
        for r, r0 in zip(rho, rho0):
            r.copy_(r0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, stats = qpr.batch_steady_state(probs, dt=a.dt, tol=a.tol, max_steps=a.max_steps,
                                           ref_refresh=a.ref_refresh, device=local)
        torch.cuda.synchronize()
        return time.perf_counter() - t, stats
    t, stats = solve()
    steps = [x["steps"] for x in stats]
    return {"workload": f"{a.batch_count} heavy-tailed graphs, N ~ U[32,1024], omega ~ U[0.1,0.95], alpha=0.85, "
                        f"rho0=I/N, RK4 dt={a.dt}, each to ||L(rho)||_F<{a.tol}",
            "time_to_steady_state_s": t, "timed": "the whole qpr_batch_steady_state call (host assembly, "
            "upload, solve, download), wall clock", "sum_n2": int(sum(g.n ** 2 for g in gs)),
            "rk4_steps_max": max(steps), "rk4_steps_mean": float(np.mean(steps)),
            "converged": int(sum(x["converged"] for x in stats)), "gpu_launches": int(stats[0]["kernel_launches"])}


def shard_time(local_total, steps, dist=None, device=None):
    """Shards (the batch split over the ranks, every rank solving its own
    problems): the batch is done when the slowest rank is, so the time per
    step is the max over ranks of the timed totals over the steps. Returns
    (seconds per step, max total)."""
    import torch

    total = float(local_total)
    if dist is not None:
        t = torch.tensor([total], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total / steps, total


def run_batch(a):
    """One step = one qpr_batch_steady_state call over the whole batch; with
    N ranks each rank solves its shard of the problems (shard.partition, no
    collective on the data path) and the step ends with the slowest rank."""
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2003_04930_gb300 import graphs, qpr, shard
    from paper_2003_04930_gb300.build import build_library
    build_library()
    specs = graphs.batch_specs(a.batch_count)
    mine = shard.partition([shard.batch_cost(n, om) for n, om, seed in specs], world)[rank]
    gs = [graphs.heavy_tailed(specs[i][0], specs[i][2]) for i in mine]
    rho0 = [torch.from_numpy(graphs.maximally_mixed(g.n)).to(dev) for g in gs]
    rho = [r.clone() for r in rho0]
    probs = [(g, specs[i][1], r) for g, i, r in zip(gs, mine, rho)]

    def solve():
        if not probs:  # more ranks than problems: this rank has none
            return qpr.QPR_OK, [{"steps": 0, "converged": 0, "kernel_launches": 0}]
        for r, r0 in zip(rho, rho0):
            r.copy_(r0)
        return qpr.batch_steady_state(probs, dt=a.dt, tol=a.tol, max_steps=a.max_steps, ref_refresh=a.ref_refresh,
                                      device=local)

    for _ in range(a.warmup):
        solve()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times, stats = [], None
    for _ in range(a.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st, stats = solve()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    value, _ = shard_time(sum(times), a.steps, dist, dev)
    steps = [s["steps"] for s in stats]
    loc = torch.tensor([max(steps), float(np.sum(steps)), len(probs), sum(s["converged"] for s in stats),
                        int(stats[0]["kernel_launches"])], dtype=torch.float64, device=dev)
    if dist is not None:
        parts = [torch.zeros_like(loc) for _ in range(world)]
        dist.all_gather(parts, loc)
        dist.destroy_process_group()
    else:
        parts = [loc]
    if rank != 0:
        return 0
    parts = [p.cpu().tolist() for p in parts]
    line = {"metric": "time-to-steady-state of the whole batch (resid 1e-8)", "value": value, "unit": "s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{a.batch_count} heavy-tailed graphs, N ~ U[32,1024], omega ~ U[0.1,0.95], "
                                   f"alpha=0.85, rho0=I/N, RK4 dt={a.dt}, tol={a.tol}",
                       "sum_n2": int(sum(n * n for n, om, seed in specs)), "ref_refresh": a.ref_refresh,
                       "parallelism": f"batch shards {world}" if world > 1 else "one batch",
                       "problems_per_rank": [int(p[2]) for p in parts]},
            "rk4_steps_max": int(max(p[0] for p in parts)),
            "rk4_steps_mean": float(sum(p[1] for p in parts) / sum(p[2] for p in parts)),
            "converged": int(sum(p[3] for p in parts)), "clocks": clocks,
            "gpu_launches": int(a.steps * sum(p[4] for p in parts))}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch":
        return run_batch(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
