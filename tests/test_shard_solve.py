"""The plan for sharding one solve over ranks (shard.partition_tile_pairs),
run as a CPU model with world_size-2 gloo process groups: each rank forms
the Lindblad right-hand side of Eq. 1 on its own tile pairs from the whole
stage input, the ranks exchange their tiles (an all-reduce of disjoint
tiles, i.e. an all-gather) and add their trace and residual partials, and
one classical RK4 step must equal the oracle's step. The GPU path of this
plan (NCCL between GB300s) is not built: every machine here has one GPU."""
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
        _, H, G, c = o.operators()
        np_ = ((N + TILE - 1) // TILE) * TILE
        mine = shard.partition_tile_pairs(np_, world, tile=TILE)[rank]
        sl = lambda t: slice(t * TILE, min((t + 1) * TILE, N))

        def gather(local):  # disjoint tiles from every rank: the all-gather of the plan
            t = torch.from_numpy(local.view(np.float64).copy())
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.numpy().view(np.complex128).reshape(N, N)

        def f_tiles(y):
            # this rank's tiles of f(y) (Eq. 1 with L_ij = sqrt(G_ij) |i><j|): the commutator from
            # X_IJ = H_I. y_.J and X_JI, the dissipator from diag(G p) and the column sums c
            k = np.zeros((N, N), dtype=np.complex128)
            gp = G @ np.real(np.diag(y))
            res = 0.0
            for i, j in mine:
                a, b = sl(i), sl(j)
                if a.start >= N or b.start >= N:
                    continue
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

        y = graphs.random_density(N, 5, rank=3)
        # residual partials of the start: ||f(y)||_F^2 summed over the ranks
        k1, r = f_tiles(y)
        rt = torch.tensor([r], dtype=torch.float64)
        dist.all_reduce(rt, op=dist.ReduceOp.SUM)
        k1 = gather(k1)
        k2 = gather(f_tiles(y + 0.5 * DT * k1)[0])
        k3 = gather(f_tiles(y + 0.5 * DT * k2)[0])
        k4 = gather(f_tiles(y + DT * k3)[0])
        yn = y + DT / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        # the trace renormalisation from the diagonal tiles' partials
        tr = sum(float(np.real(np.trace(yn[sl(i), sl(i)]))) for i, j in mine if i == j and sl(i).start < N)
        tt = torch.tensor([tr], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        yn = yn / float(tt.item())
        ref = o.evolve(y, DT, 1)
        out[rank] = (float(np.abs(yn - ref).max()), float(np.sqrt(rt.item())), o.residual(y),
                     float(np.abs(k1 - o.rhs(y)).max()))
    finally:
        dist.destroy_process_group()


def test_sharded_rk4_step_equals_the_oracle():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, 29781, out), nprocs=world, join=True)
    for r in range(world):
        step_err, resid, resid_ref, rhs_err = out[r]
        assert rhs_err <= 1e-13
        assert step_err <= 1e-14
        assert resid == pytest.approx(resid_ref, rel=1e-12)
