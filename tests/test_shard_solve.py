"""The plan for sharding one solve over ranks (shard.partition_tile_pairs),
run as a CPU model with world_size-2 gloo process groups on the padded
layout of the GPU forms: each rank forms the Lindblad right-hand side of
Eq. 1 on its own tile pairs from the whole stage input, the ranks all-gather
the tiles they wrote (each placing the others' by the plan) and add their
trace and residual partials. One classical RK4 step must equal the oracle's
step, the padding must stay zero, and the bytes each rank receives must be
those shard.stage_exchange_bytes gives. The GPU path of this plan (NCCL
between GB300s) is not built: every machine here has one GPU."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2003_04930_gb300 import graphs, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, OMEGA, ALPHA, DT, TILE = 70, 0.7, 0.85, 0.01, 16


def test_tile_pair_plan_covers_every_pair_once():
    for world in (1, 2, 3, 5):
        parts = shard.partition_tile_pairs(96, world, tile=16)
        flat = sorted(p for part in parts for p in part)
        assert flat == [(i, j) for i in range(6) for j in range(i, 6)]
        loads = [sum(1 if i == j else 2 for i, j in part) for part in parts]
        assert max(loads) - min(loads) <= 2
    # all-gather volume: each rank receives the tiles it did not write
    b = shard.stage_exchange_bytes(96, 2, tile=16, element_bytes=8)
    assert sum(b) == (36 - 0) * 16 * 16 * 8 and all(x > 0 for x in b)


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    from oracle import Oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = graphs.heavy_tailed(N, 12)
        o = Oracle.from_edges(g, alpha=ALPHA, omega=OMEGA)
        _, H0, G0, c0 = o.operators()
        # the padded layout of the GPU forms: np_ a multiple of the tile, zero rows and columns beyond N
        np_ = ((N + TILE - 1) // TILE) * TILE
        H = np.zeros((np_, np_)); H[:N, :N] = H0
        G = np.zeros((np_, np_)); G[:N, :N] = G0
        c = np.zeros(np_); c[:N] = c0
        parts = shard.partition_tile_pairs(np_, world, tile=TILE)
        mine = parts[rank]
        sl = lambda t: slice(t * TILE, (t + 1) * TILE)

        def written(pairs):  # the tiles a rank writes, in its order: (I, J) and the mirror (J, I)
            return [t for i, j in pairs for t in ([(i, j)] if i == j else [(i, j), (j, i)])]

        owned = [written(p) for p in parts]
        slots = max(len(t) for t in owned)

        def gather(kpad):
            # the plan's all-gather: every rank sends the tiles it wrote (padded to a common count)
            # and places every other rank's tiles by the plan; returns the whole matrix and the
            # bytes of tiles this rank received
            buf = np.zeros((slots, TILE, TILE), dtype=np.complex128)
            for q, (i, j) in enumerate(owned[rank]):
                buf[q] = kpad[sl(i), sl(j)]
            t = torch.from_numpy(buf.view(np.float64).copy())
            bufs = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(bufs, t)
            full = np.zeros((np_, np_), dtype=np.complex128)
            received = 0
            for r in range(world):
                b = bufs[r].numpy().view(np.complex128)
                for q, (i, j) in enumerate(owned[r]):
                    full[sl(i), sl(j)] = b[q]
                if r != rank:
                    received += len(owned[r]) * TILE * TILE * 16
            return full, received

        def f_tiles(y):
            # this rank's tiles of f(y) (Eq. 1 with L_ij = sqrt(G_ij) |i><j|): the commutator from
            # X_IJ = H_I. y_.J and X_JI, the dissipator from diag(G p) and the column sums c
            k = np.zeros((np_, np_), dtype=np.complex128)
            gp = G @ np.real(np.diag(y))
            res = 0.0
            for i, j in mine:
                a, b = sl(i), sl(j)
                xij = H[a, :] @ y[:, b]
                xji = H[b, :] @ y[:, a]
                kij = -1j * (1 - OMEGA) * (xij - xji.conj().T) - OMEGA * 0.5 * (c[a][:, None] + c[b][None, :]) * y[a, b]
                if i == j:
                    kij = kij + OMEGA * np.diag(gp[a])
                k[a, b] = kij
                res += (1.0 if i == j else 2.0) * float(np.sum(np.abs(kij) ** 2))
                if i != j:
                    k[b, a] = kij.conj().T
            return k, res

        y0 = graphs.random_density(N, 5, rank=3)
        y = np.zeros((np_, np_), dtype=np.complex128); y[:N, :N] = y0
        # residual partials of the start: ||f(y)||_F^2 summed over the ranks
        k1, r = f_tiles(y)
        rt = torch.tensor([r], dtype=torch.float64)
        dist.all_reduce(rt, op=dist.ReduceOp.SUM)
        k1, received = gather(k1)
        k2 = gather(f_tiles(y + 0.5 * DT * k1)[0])[0]
        k3 = gather(f_tiles(y + 0.5 * DT * k2)[0])[0]
        k4 = gather(f_tiles(y + DT * k3)[0])[0]
        yn = y + DT / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        # the trace renormalisation from the diagonal tiles' partials
        tr = sum(float(np.real(np.trace(yn[sl(i), sl(i)]))) for i, j in mine if i == j)
        tt = torch.tensor([tr], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        yn = yn / float(tt.item())
        ref = o.evolve(y0, DT, 1)
        plan_bytes = shard.stage_exchange_bytes(np_, world, tile=TILE, element_bytes=16)[rank]
        out[rank] = (float(np.abs(yn[:N, :N] - ref).max()), float(np.sqrt(rt.item())), o.residual(y0),
                     float(np.abs(k1[:N, :N] - o.rhs(y0)).max()), float(np.abs(yn[N:, :]).max(initial=0.0)),
                     received, plan_bytes)
    finally:
        dist.destroy_process_group()


def test_sharded_rk4_step_equals_the_oracle():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, 29781, out), nprocs=world, join=True)
    for r in range(world):
        step_err, resid, resid_ref, rhs_err, pad, received, plan_bytes = out[r]
        assert rhs_err <= 1e-13
        assert step_err <= 1e-14
        assert resid == pytest.approx(resid_ref, rel=1e-12)
        assert pad == 0.0  # the padding stays zero
        assert received == plan_bytes > 0  # the exchange moves what the plan says
