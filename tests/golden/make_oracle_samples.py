"""Writes tests/golden/oracle_samples.json: seeded samples of the CPU oracle's DD-PCG results on
problems whose subdomains are too large for the oracle to finish inside a GPU test run.

Only the oracle (oracle/) and the workload parameters (sg_workloads) are used.  For each case the
oracle advances `steps` Newmark steps twice, at PCG tolerance 1e-13 (the FP64 parity setting) and
at the case's workload tolerance, and records per run: the outer iteration counts per step, the
l2 norm of every PCE mode of U over the free nodes, and the values of U at a sample of
(free node, mode) entries: half drawn uniformly (numpy default_rng, seed 20251227, per case), half
the entries of largest magnitude of the tight run's field (where the wave is).  The GPU tests
compare the library's fields at the same entries.

Cases:
  l65_m5p2   128^2 grid, 2 x 2 subdomains (65 x 65 nodes each), KL M = 5, PCE order 2 (P = 21),
             sigma 0.3, correlation length 0.1: the 1024^2 workload's PCE sizes and field.
  l65_m4p3   the same grid with M = 4, order 3 (P = 35), sigma 0.4, correlation length 0.2: the
             512^2 workload's.
  b240       the widest 2 x 2 batch instance with P = 10 (240^2 grid, 121 x 121-node subdomains).

Run: python tests/golden/make_oracle_samples.py  (about 20 minutes on 8 x86 cores; SuperLU runs
single-threaded).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sg_workloads as w  # noqa: E402
from oracle import dd, sg  # noqa: E402

NSAMPLE = 2048


def cases():
    c5 = w.config("ricker1024")
    c3 = w.config("ricker512")
    yield "l65_m5p2", c5.replace(name="l65_m5p2", N=128, s=2, dt=w.cfl_dt(128)), 6
    yield "l65_m4p3", c3.replace(name="l65_m4p3", N=128, s=2, dt=w.cfl_dt(128)), 6
    wide = [p for p in w.batch_problems(256) if p.s == 2 and p.N == 240]
    yield "b240", wide[0], 6


def run(prob, steps, tol):
    sgp = sg.SGProblem(prob)
    d = dd.DDSolver(prob)
    U, _, _, it = dd.run_dd(sgp, d, steps, tol=tol)
    return U.reshape(-1, prob.P), [int(i) for i, _ in it]


def main(only=None):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_samples.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name, prob, steps in cases():
        if only and name not in only:
            continue
        t0 = time.time()
        rng = np.random.default_rng(20251227)
        nf = (prob.N - 1) ** 2
        runs = {label: run(prob, steps, tol) for label, tol in (("tight", 1e-13), ("workload", prob.tol))}
        flat = np.argsort(-np.abs(runs["tight"][0]).ravel(), kind="stable")[: NSAMPLE // 2]
        node = np.concatenate([rng.integers(0, nf, NSAMPLE // 2), flat // prob.P])
        mode = np.concatenate([rng.integers(0, prob.P, NSAMPLE // 2), flat % prob.P])
        rec = {"problem": {k: getattr(prob, k) for k in ("N", "s", "M", "p", "p_in", "sigma", "bx", "by", "g0", "dt",
                                                          "tol", "alpha0", "alpha1")},
               "source": {k: getattr(prob.source, k) for k in ("kind", "x0", "y0", "width", "freq", "amp")},
               "steps": steps, "n_uniform": NSAMPLE // 2, "node": node.tolist(), "mode": mode.tolist()}
        for label, tol in (("tight", 1e-13), ("workload", prob.tol)):
            U, its = runs[label]
            rec[label] = {"tol": tol, "iters": its, "mode_norm": np.linalg.norm(U, axis=0).tolist(),
                          "norm": float(np.linalg.norm(U)), "values": U[node, mode].tolist()}
        out[name] = rec
        json.dump(out, open(path, "w"), separators=(",", ":"))
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
