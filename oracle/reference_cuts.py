"""FP64 oracle best cuts of the benchmark's workloads at fixed seeds.

TEST INFRASTRUCTURE ONLY: a standalone script that runs the CPU oracle
(oracle/deco_oracle.py) on the same seeded graphs, starting points and phase
schedules as the benchmark, so that the cut gap of the FP32 and BF16 kernels
against FP64 arithmetic can be stated per workload.  It calls nothing but the
oracle and the seeded generators in graphgen/.  The runs take minutes (main
workload) to about an hour (the 10^6-node graph, one thread).

  python -m oracle.reference_cuts main | er1m | dense | learned
"""
from __future__ import annotations

import json
import sys
import time

import graphgen as gg

from . import deco_oracle as O

MAIN_SCHEDULE = [O.Phase(1, 800, 0.01, 0.9), O.Phase(2, 200, 0.001, 0.9)] * 2


def _run(name, g, B, phases, params, seed):
    t0 = time.time()
    r = O.solve(g, B, phases, params, seed)
    print(json.dumps({"workload": name, "n": g.n, "m": g.m, "B": B, "seed": seed, "best_cut": r.best_cut,
                      "phase_best_cuts": [int(c.max()) for c in r.phase_cuts],
                      "seconds": round(time.time() - t0, 1)}), flush=True)


def main(which: str):
    if which == "main":
        # ER(800, 0.06) seed 1 and the 40 x 20 +-1 torus seed 2; B = 1024, starts
        # [0, 512) IDI-centred and [512, 1024) uniform; pDECO 2 x (800 + 200 lifted)
        p = O.Params(init="idi_half_uniform")
        _run("er800", gg.er_graph(800, 0.06, 1), 1024, MAIN_SCHEDULE, p, 7)
        _run("torus40x20", gg.torus_graph(40, 20, 2), 1024, MAIN_SCHEDULE, p, 7)
    elif which == "er1m":
        # ER(10^6, average degree 10) seed 4; B = 128 IDI starts; T = 1000, alpha = 0.01
        _run("er1m", gg.er_graph_avg_degree(1_000_000, 10, 4), 128, [O.Phase(1, 1000, 0.01, 0.0)],
             O.Params(init="idi"), 2)
    elif which == "dense":
        # ER(4096, 0.5) seed 4096; B = 128 IDI starts; T = 1000, alpha = 1e-4
        _run("er4096", gg.er_graph(4096, 0.5, 4096), 128, [O.Phase(1, 1000, 1e-4, 0.0)], O.Params(init="idi"), 2)
    elif which == "learned":
        # the learned proposal's evaluation graphs: the long IDI run that defines the target
        sched = [O.Phase(1, 1000, 0.02, 0.9), O.Phase(2, 250, 0.002, 0.9)] * 4
        _run("ba2000_m4", gg.ba_graph(2000, 4, 9001), 256, sched, O.Params(init="idi"), 31337)
        _run("er5000_p0.002", gg.er_graph(5000, 0.002, 9002), 256, sched, O.Params(init="idi"), 31337)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
