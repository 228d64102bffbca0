"""FP64 oracle best cuts of the benchmark's workloads at fixed seeds.

TEST INFRASTRUCTURE ONLY: a standalone script that runs the CPU oracle
(oracle/deco_oracle.py) on the same seeded graphs, starting points and phase
schedules as the benchmark, so that the cut gap of the FP32 and BF16 kernels
against FP64 arithmetic can be stated per workload.  It calls nothing but the
oracle and the seeded generators in graphgen/.  The runs take minutes (main
workload) to about an hour (the 10^6-node graph, one thread).

  python -m oracle.reference_cuts main | er1m | dense | learned | batch16 [--write]

With --write the lines also go to tests/golden/reference_cuts_<workload>.jsonl
(the stored FP64 values the tests and the design notes compare the kernels'
best cuts with).
"""
from __future__ import annotations

import json
import os
import sys
import time

import graphgen as gg

from . import deco_oracle as O

MAIN_SCHEDULE = [O.Phase(1, 800, 0.01, 0.9), O.Phase(2, 200, 0.001, 0.9)] * 2
GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
_out = None


def _run(name, g, B, phases, params, seed):
    t0 = time.time()
    r = O.solve(g, B, phases, params, seed)
    line = json.dumps({"workload": name, "n": g.n, "m": g.m, "B": B, "seed": seed, "best_cut": r.best_cut,
                       "best_init": r.best_init, "best_phase": r.best_phase,
                       "phase_best_cuts": [int(c.max()) for c in r.phase_cuts],
                       "schedule": [[p.lift, p.steps, p.alpha, p.momentum] for p in phases],
                       "init": params.init, "seconds": round(time.time() - t0, 1)})
    print(line, flush=True)
    if _out is not None:
        _out.write(line + "\n")
        _out.flush()


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
    elif which == "batch16":
        # the first 16 graphs of the 256-graph family (BA, n ~ U{200..1200},
        # m = 4, seeds 3000 + i): batched pDECO with the population search,
        # B = 256, 32 candidates x 8 starts, 5 rounds alternating lift 1 / 2,
        # T ~ U{500..2000}, e ~ U[-4, -1], momentum 0.9, IDI + uniform starts
        import numpy as np
        rng = np.random.default_rng(3000)
        sizes = rng.integers(200, 1201, 256)[:16]
        graphs = [gg.ba_graph(int(nn), 4, 3000 + i) for i, nn in enumerate(sizes)]
        t0 = time.time()
        r = O.solve_batch_population(graphs, 256, 32, 5, [1, 2], 500, 2000, -4.0, -1.0, 0.9,
                                     O.Params(init="idi_half_uniform"), 2)
        line = json.dumps({"workload": "ba16_population", "n": [g.n for g in graphs], "m": [g.m for g in graphs],
                           "B": 256, "candidates": 32, "rounds": 5, "lifts": [1, 2], "t_range": [500, 2000],
                           "e_range": [-4.0, -1.0], "momentum": 0.9, "init": "idi_half_uniform", "seed": 2,
                           "best_cuts": [int(c) for c in r.best_cuts],
                           "round_scores": [[int(x) for x in sc] for sc in r.round_scores],
                           "final_T": [int(x) for x in r.final_T], "seconds": round(time.time() - t0, 1)})
        print(line, flush=True)
        if _out is not None:
            _out.write(line + "\n")
            _out.flush()
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else ""
    if "--write" in sys.argv[2:]:
        _out = open(os.path.join(GOLDEN, f"reference_cuts_{which}.jsonl"), "w")
    main(which)
