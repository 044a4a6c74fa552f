"""Time the oracle's SG-DD step on a workload (CPU baseline; test infrastructure only).

Runs the oracle as it stands: set-up (not timed), `warmup` untimed steps, then `steps` timed
steps; prints one JSON line {"steps_per_s", "steps", "seconds", "setup_s", "iters"}.
Thread count is whatever the caller's environment allows (bench.py pins BLAS to 1 thread).
"""
import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import sg_workloads as w  # noqa: E402
from oracle import dd, sg  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="ricker128")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=0)
    a = ap.parse_args()
    prob = w.config(a.config)
    t0 = time.perf_counter()
    sgp = sg.SGProblem(prob)
    d = dd.DDSolver(prob)
    setup = time.perf_counter() - t0
    state = None
    if a.warmup:
        U, V, A, _ = dd.run_dd(sgp, d, a.warmup)
        state = (U, V, A, a.warmup)
    t0 = time.perf_counter()
    _, _, _, it = dd.run_dd(sgp, d, a.steps, state=state)
    sec = time.perf_counter() - t0
    print(json.dumps({"steps_per_s": a.steps / sec, "steps": a.steps, "seconds": sec, "setup_s": setup,
                      "iters": [i for i, _ in it]}))


if __name__ == "__main__":
    main()
