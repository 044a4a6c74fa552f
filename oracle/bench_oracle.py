"""Time the oracle's SG-DD step on a workload (CPU baseline; test infrastructure only).

Two modes, both running the oracle as it stands:

* full (default): set-up (not timed), `warmup` untimed steps, then `steps` timed steps of
  dd.run_dd; prints {"steps_per_s", "steps", "seconds", "setup_s", "iters", "mode": "full"}.
* sampled (--sample): for workloads whose 256 subdomain factorisations would take hours, each
  worker process builds the local operators of ONE subdomain (DDSolver with `subs`) and times the
  oracle's own per-subdomain operations of one SG-DD step with `n_outer` PCG iterations (Alg. 1,
  Sec. 5): the local effective load, the condensed right-hand side (one interior solve), n_outer + 1
  local Schur-complement applications (one interior solve each), n_outer local Neumann solves with
  their corner products and coarse extension, and the interior recovery (one interior solve).  The
  step's global work is timed once on full-size vectors: the Newmark predictor and update on every
  SG unknown, and n_outer coarse solves with a dense Cholesky factor of the coarse size.  Per-step
  time on one core: nsub x t_sub + t_global; on W workers (one subdomain each, in parallel, one
  thread each): (nsub / W) x max t_sub + t_global.  Prints {"steps_per_s" (all workers),
  "steps_per_s_1core", "workers", "t_sub", "t_global", "setup_s", "mode": "sampled"}.
Thread count is whatever the caller's environment allows (bench.py pins BLAS to 1 thread).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

import sg_workloads as w  # noqa: E402
from oracle import dd, sg  # noqa: E402


def sample_subdomain_step(d, L, F_glob, um, uc, n_outer, rng):
    """The oracle's local operations of one SG-DD step on subdomain L (same calls as
    DDSolver.solve_step / pcg / precond make for one subdomain)."""
    f = d.local_load(L, F_glob, um, uc)
    gs = f[L["Gam"]].copy()
    if L["I"].size:
        gs -= L["Kt"][L["Gam"]][:, L["I"]] @ d.solve_I(L, f[L["I"]])
    x = rng.standard_normal(L["Gam"].size)
    for _ in range(n_outer + 1):
        x = 0.5 * x + 1e-3 * d.schur_local(L, x)
    for _ in range(n_outer):
        wv = L["D"] * x
        y, t = d.neumann(L, wv[L["Gr"]])
        if L["c"].size:
            _ = L["Kt"][L["c"]][:, L["ir"]] @ d._ir_vec(L, y, t)
            _ = L["Phi"] @ rng.standard_normal(L["c"].size)
    if L["I"].size:
        _ = d.solve_I(L, f[L["I"]] - L["Kt"][L["I"]][:, L["Gam"]] @ x)
    return gs


def _coarse_basis(d, L):
    """Phi_s of the sampled subdomain (Eq. Fcc_2 column solves), as the oracle's set-up builds it."""
    Kt = L["Kt"]
    Kir_c = Kt[L["ir"]][:, L["c"]].toarray()
    Phi = np.zeros((L["r"].size, L["c"].size))
    for col in range(L["c"].size):
        v = -L["lu_N"].solve(Kir_c[:, col])
        Phi[:, col] = v[L["ir_r"]]
    L["Phi"] = Phi


def worker(args):
    config, sub_index, n_outer, reps = args
    prob = w.config(config)
    t0 = time.perf_counter()
    d = dd.DDSolver(prob, subs=[sub_index])
    L = d.loc[0]
    _coarse_basis(d, L)
    nfree = d.part.free.size
    rng = np.random.default_rng(sub_index)
    F = rng.standard_normal(nfree * d.P)
    um = rng.standard_normal(nfree * d.P)
    uc = rng.standard_normal(nfree * d.P)
    setup = time.perf_counter() - t0
    sample_subdomain_step(d, L, F, um, uc, n_outer, rng)  # untimed first pass
    ts = []
    for _ in range(reps):
        t1 = time.perf_counter()
        sample_subdomain_step(d, L, F, um, uc, n_outer, rng)
        ts.append(time.perf_counter() - t1)
    return {"sub": sub_index, "t_sub": float(np.median(ts)), "setup_s": setup}


def global_step_time(prob, n_outer, reps=2):
    """Newmark predictor / update on every SG unknown and n_outer coarse solves (sizes of prob)."""
    import scipy.linalg as sla
    nfree = (prob.N - 1) ** 2
    n = nfree * prob.P
    rng = np.random.default_rng(1)
    U, V, A, Un = (rng.standard_normal(n) for _ in range(4))
    nc = (prob.s - 1) ** 2 * prob.P
    B = rng.standard_normal((nc, nc)) / np.sqrt(nc)
    Fcc = B @ B.T + np.eye(nc)
    cho = sla.cho_factor(Fcc)
    dvec = rng.standard_normal(nc)
    dt = prob.dt
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        um = (U + dt * V) / (sg.ZETA * dt * dt) + (1.0 - 2.0 * sg.ZETA) * A / (2.0 * sg.ZETA)
        uc = sg.GAMMA * dt * um - V - (1.0 - sg.GAMMA) * A * dt
        An = Un / (sg.ZETA * dt * dt) - um
        Vn = V + dt * ((1.0 - sg.GAMMA) * A + sg.GAMMA * An)
        for _ in range(n_outer):
            sla.cho_solve(cho, dvec)
        ts.append(time.perf_counter() - t0)
        del uc, Vn
    return float(np.median(ts))


def sampled(config, workers, n_outer, reps):
    prob = w.config(config)
    s = prob.s
    # interior subdomains nearest the centre first (every class of node present)
    order = sorted(range(s * s), key=lambda k: (abs(k % s - (s - 1) / 2) + abs(k // s - (s - 1) / 2), k))
    subs = order[:workers]
    t0 = time.perf_counter()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(worker, [(config, k, n_outer, reps) for k in subs])
    wall = time.perf_counter() - t0
    t_glob = global_step_time(prob, n_outer)
    tsub = [r["t_sub"] for r in res]
    nsub = s * s
    t1 = nsub * float(np.median(tsub)) + t_glob
    tall = (nsub / workers) * max(tsub) + t_glob
    return {"mode": "sampled", "steps_per_s": 1.0 / tall, "steps_per_s_1core": 1.0 / t1, "workers": workers,
            "t_sub": tsub, "t_global": t_glob, "n_outer": n_outer, "nsub": nsub, "setup_s": max(r["setup_s"] for r in res),
            "wall_s": wall, "subdomains": subs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="ricker128")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--sample", action="store_true")
    ap.add_argument("--workers", type=int, default=1)
    ap.add_argument("--n-outer", type=int, default=4)
    a = ap.parse_args()
    if a.sample:
        print(json.dumps(sampled(a.config, max(1, a.workers), a.n_outer, max(1, a.steps))))
        return
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
    print(json.dumps({"mode": "full", "steps_per_s": a.steps / sec, "steps": a.steps, "seconds": sec, "setup_s": setup,
                      "iters": [i for i, _ in it]}))


if __name__ == "__main__":
    main()
