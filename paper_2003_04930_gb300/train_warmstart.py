"""Train the warm-start network on solver-generated steady states.

    python -m paper_2003_04930_gb300.train_warmstart [--count 256] [--n-hi 1024] [--epochs 60] [--out PATH]

Labels come from the batched solver (qpr_batch_steady_state, tol 1e-6) on
`--count` seeded heavy-tailed graphs (warmstart.training_specs: seeds 10000 +
i, N ~ U[64, n_hi], omega ~ U[0.1, 0.95]); the network is trained with the
library's own forward/backward/Adam kernels (qpr_gnn_train). The flat FP32
parameter vector is saved with numpy.save (default: data/warmstart_gnn.npy in
this package), where bench.py and warmstart.load_network look for it.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "warmstart_gnn.npy")


def main():
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2003_04930_gb300 import qpr as Q
    from paper_2003_04930_gb300 import warmstart
    from paper_2003_04930_gb300.build import build_library

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--n-hi", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", default=DEFAULT_OUT)
    a = ap.parse_args()
    build_library()
    t0 = time.time()
    data = warmstart.make_dataset(warmstart.training_specs(a.count, n_lo=64, n_hi=a.n_hi))
    t1 = time.time()
    net = Q.Gnn(seed=3)
    losses = net.train(data, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    t2 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, net.get_params())
    print(json.dumps({"out": a.out, "graphs": a.count, "labels_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
                      "loss_first": float(losses[0]), "loss_last": float(losses[-1])}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
