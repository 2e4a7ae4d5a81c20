"""Write tests/golden/oracle_steady_n922.json with the CPU oracle only.

For the airline-sized workload (heavy-tailed graph, N = 922, seed 1,
alpha = 0.85, rho0 = I/N, classical RK4 with dt = 0.01, stop at the first
step index with ||f(rho_n)||_F < 1e-8) and each omega in {0.2, 0.5, 0.8, 1.0}
it stores the oracle's step count, final residual and populations.

Usage: python tests/golden/make_oracle_steady_states.py [omega ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from oracle.cpu import populations  # noqa: E402
from paper_2003_04930_gb300 import graphs  # noqa: E402

OUT = os.path.join(HERE, "oracle_steady_n922.json")


def main(omegas):
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    g = graphs.heavy_tailed(922, 1)
    for om in omegas:
        o = Oracle.from_edges(g, alpha=0.85, omega=om)
        t = time.time()
        y, steps, r, st = o.steady_state(graphs.maximally_mixed(922), 0.01, 1e-8, 400000)
        assert st == 0, st
        data[str(om)] = {"steps": steps, "residual": r, "oracle_seconds": time.time() - t,
                         "populations": [float(x) for x in populations(y)]}
        data["workload"] = ("heavy_tailed(922, seed=1), alpha=0.85, rho0=I/N, RK4 dt=0.01, "
                            "stop at first ||f||_F < 1e-8; written by make_oracle_steady_states.py "
                            "from the CPU oracle")
        json.dump(data, open(OUT, "w"), indent=0)
        print(om, steps, r, flush=True)


if __name__ == "__main__":
    main([float(x) for x in sys.argv[1:]] or [0.8, 1.0, 0.5, 0.2])
