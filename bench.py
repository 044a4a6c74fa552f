#!/usr/bin/env python
"""Benchmark: SG-DD time steps per second on one GB300 (or N independent replicas).

Default workload (`ricker1024`): 1024 x 1024 grid (~1.05M nodes), 16 x 16 subdomains of 65 x 65
nodes, KL with M = 5 random variables, Hermite PCE order 2 (P = 21 terms, ~22M stochastic unknowns),
sigma 0.3, correlation length 0.1, Ricker source (10 Hz) at (0.3, 0.5), dt from CFL 0.65, PCG
relative residual 1e-8.  A "step" is one Newmark time step: effective load, condensed interface
RHS, interface PCG with the two-level Neumann-Neumann preconditioner, interior recovery and
Newmark update, all on the GPU.

Which steps are timed: the per-step cost grows while the wave field spreads over the subdomains
(subdomain problems with a vanishing right-hand side are skipped); from about step 200 every
subdomain carries it.  The run is therefore fast-forwarded untimed (--forward, 200 steps at this
workload) before the W warm-up steps and the K timed steps, so the number reported is the
all-subdomains-active cost that dominates the workload's 1000 steps.  The plain FP64 solver and the
end-to-end leg start from the same state.

Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on the solver's stream; a
256 MB buffer is written between timed steps (the working set, ~14 GB, is larger than L2 anyway).
The headline is the optimised solver (FP32 subdomain solves + FP64 outer PCG, one CUDA graph per
step); the plain FP64 solver is measured beside it on the same GPU.  Under torchrun each rank runs
an independent replica (weak scaling, no data-path collective); value = steps of all ranks / max
over ranks of the timed duration.

--impl reference times the FP64 CPU oracle (the reference arm of this workload) on the host.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SG-DD time-steps/sec & PCG iters vs plain FP64 DD-PCG at rel resid 1e-8"

# DRAM traffic (read + write bytes per launch) of the dominant kernel from one ncu capture, keyed by
# the sha256 prefix of that kernel's source regions (KERNEL_REGIONS) it was taken on; any other source
# reports null.  The value is k_line_w<float> at the 1024^2 workload from step 202 (every subdomain
# active), the mean of three iterate launches: 1,018,883,840 B read + 330,724,267 B written
# (profiles/k_line_w_ricker1024_dram.md).
KERNEL_TRAFFIC = {"74f2ba0e6b1026f5": 1349608107}
# source regions of the dominant kernel that the traffic figure is keyed to: k_line_w and the FP32
# partial-sum helpers it uses
KERNEL_REGIONS = (("// Mean-operator line solve fused with the inner CG update, register-tiled form",
                   "// Line sweeps of the mean-operator preconditioner with the per-line products"),
                  ("// FP32 partial sums at any magnitude", "// Division by a runtime constant"))


def kernel_source_sha():
    """sha256 prefix of the dominant kernel's source regions (the traffic figure is valid for them)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_kernels.cuh")).read()
    h = hashlib.sha256()
    for r0, r1 in KERNEL_REGIONS:
        a = src.index(r0)
        h.update(src[a:src.index(r1, a)].encode())
    return h.hexdigest()[:16]
L2_FLUSH_BYTES = 256 << 20


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself without one):
    every replica-parallel duration is reported as the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(prob, precision):
    return {"workload": prob.name, "grid": f"{prob.N}x{prob.N}", "nodes": (prob.N + 1) ** 2,
            "subdomains": f"{prob.s}x{prob.s}", "kl_M": prob.M, "pce_order": prob.p, "pce_terms": prob.P,
            "sigma": prob.sigma, "corr_len": prob.bx, "dt": prob.dt, "tol": prob.tol,
            "precision": precision, "l2": "flushed between timed steps (256 MB write)"}


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus = bus_id
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.bus is not None and self.bus.lower() not in f[1].lower():
                continue
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for n, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm), "reasons": sorted(reasons)}


def bus_id_of(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# workloads whose oracle set-up (one sparse LU per subdomain) is out of reach on the host: the CPU
# baseline times a per-subdomain sample of the oracle's step and scales it by the subdomain count
SAMPLED = {"ricker512", "ricker1024", "ricker1024q"}
# untimed steps before the warm-up: the point from which every subdomain carries the wave field
FORWARD = {"ricker1024": 200, "ricker512": 200, "ricker1024q": 200}


def cpu_workers():
    return max(1, (os.cpu_count() or 2) - 2)


def start_cpu_baseline(cfg, steps, n_outer=4):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.join(ROOT, "oracle", "bench_oracle.py"), "--config", cfg, "--steps", str(steps)]
    if cfg in SAMPLED:
        cmd += ["--sample", "--workers", str(cpu_workers()), "--n-outer", str(n_outer)]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)


def cpu_baseline_line(d, cfg, steps):
    """cpu_baseline object of the JSON line from bench_oracle.py's output."""
    if d.get("mode") == "sampled":
        return {"value": d["steps_per_s"], "unit": "steps/s", "cores": d["workers"], "kind": "oracle",
                "one_core": d["steps_per_s_1core"], "nproc": os.cpu_count(),
                "sample": (f"{cfg}: {d['workers']} worker processes (one thread each) each build the oracle's "
                           f"local operators of one subdomain and time its per-subdomain operations of one "
                           f"SG-DD step with {d['n_outer']} PCG iterations (median {steps} repetitions; "
                           f"t_sub = {min(d['t_sub']):.2f}-{max(d['t_sub']):.2f} s); the step's global "
                           f"vector and coarse work is timed once ({d['t_global']:.2f} s); steps/s = "
                           f"1 / ({d['nsub']} / workers x max t_sub + t_global), one core: "
                           f"1 / ({d['nsub']} x median t_sub + t_global); set-up ({d['setup_s']:.0f} s) "
                           f"not timed, FP64 numpy/scipy, sparse LU subdomain solves"),
                "seconds": d["wall_s"]}
    return {"value": d["steps_per_s"], "unit": "steps/s", "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
            "sample": f"{steps} time steps of {cfg} after the oracle's untimed set-up "
                      f"({d['setup_s']:.0f} s), FP64 numpy/scipy, BLAS pinned to 1 thread",
            "seconds": d["seconds"]}


def finish_cpu_baseline(proc, cfg, steps, timeout):
    if proc is None:
        return None
    try:
        out, err = proc.communicate(timeout=timeout)
        return cpu_baseline_line(json.loads(out.strip().splitlines()[-1]), cfg, steps)
    except Exception as e:  # a missing baseline is reported, never invented
        proc.kill()
        return {"value": None, "unit": "steps/s", "cores": None, "kind": "oracle", "sample": f"failed: {e}"}


def tc_product_shape(prob):
    L = prob.N // prob.s + 1
    Kp = -(-L * L // 128) * 128
    NB = 16 if prob.P <= 16 else 32
    return L, prob.s * prob.s, Kp, NB


def tc_product_bytes(prob):
    """Algorithmic bytes of one tensor-core preconditioner launch over all subdomains: the BF16
    dense inverse of the mean operator (nsub x Kp^2 x 2 B, read once), the packed residual image
    (nsub x Kp rows x [hi; lo] NB modes x 2 B) and z written + r read (2 FP32 vector passes)."""
    L, nsub, Kp, NB = tc_product_shape(prob)
    return nsub * Kp * Kp * 2 + nsub * Kp * 2 * NB * 2 + 2 * nsub * L * L * prob.P * 4


def tc_product_flops(prob):
    """Tensor-core flops of one launch: D[Kp x 2 NB] = Ainv[Kp x Kp] [r_hi; r_lo]^T per subdomain."""
    L, nsub, Kp, NB = tc_product_shape(prob)
    return 2 * nsub * Kp * Kp * 2 * NB


def line_kernel_bytes(prob, tsize):
    """Algorithmic bytes of one fused line-solve launch over all subdomains (every subdomain problem
    active): the CG update reads r, x, p, q and writes x, r (6 vector passes), the preconditioned
    residual z is written (1 pass), and the line factors S_j^{-1} of every subdomain are read once
    (L^3 values).  The kernel's own extra traffic (the factor read once per sweep, rows padded to a
    multiple of 4, and y parked in z between the sweeps) is not counted."""
    L = prob.N // prob.s + 1
    nvec = prob.s * prob.s * L * L * prob.P
    return 7 * nvec * tsize + prob.s * prob.s * L ** 3 * tsize


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host's cores, rank 0 only.  Workloads
    whose oracle set-up is out of reach (one sparse LU per subdomain, hours at 1024^2) are timed on a
    per-subdomain sample of the oracle's step, one subdomain per worker process, scaled by the
    subdomain count (oracle/bench_oracle.py --sample)."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return 0
    import sg_workloads as w
    prob = w.config(args.config)
    steps = max(1, min(args.steps, 3))
    warm = min(args.warmup, 1)
    if args.config in SAMPLED:
        from oracle import bench_oracle
        d = bench_oracle.sampled(args.config, cpu_workers(), 4, steps)
        v = d["steps_per_s"]
        cpu = cpu_baseline_line(d, args.config, steps)
        its = 4.0
        sec = steps / v
    else:
        from oracle import dd, sg
        sgp = sg.SGProblem(prob)
        dds = dd.DDSolver(prob)
        state = None
        if warm:
            U, V, A, _ = dd.run_dd(sgp, dds, warm)
            state = (U, V, A, warm)
        t0 = time.perf_counter()
        _, _, _, it = dd.run_dd(sgp, dds, steps, state=state)
        sec = time.perf_counter() - t0
        v = steps / sec
        its = sum(i for i, _ in it) / len(it)
        cpu = {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{steps} time steps after {warm} warm-up step(s); FP64 numpy/scipy oracle "
                         f"as it stands (sparse LU subdomain solves), one process"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * sec / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(prob, "fp64 (CPU oracle)"), l2="not applicable (host CPU)"),
            "pcg_iters_per_step": its, "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched workload: independent problems of uneven size advanced together, one graph launch per
    time step for the whole batch (mixed precision, autotuned tiles, learned warm start unless
    --batch-warm prev)."""
    import torch
    import sg_workloads as w
    from paper_2512_23027_gb300 import Solver, solve_batch
    from paper_2512_23027_gb300.binding import SG_MIXED, SG_WARM_LEARNED, SG_WARM_PREV
    from paper_2512_23027_gb300.binding import SGError
    drawn = w.batch_problems(256)[: args.batch]
    warm = SG_WARM_PREV if args.batch_warm == "prev" else SG_WARM_LEARNED
    t0 = time.perf_counter()
    probs, solvers, skipped = [], [], []
    for p in drawn:
        try:
            solvers.append(Solver(p, precision=SG_MIXED, autotune=True, warm=warm))
            probs.append(p)
        except SGError as e:  # reported, never silently replaced
            if e.code != -7:
                raise
            skipped.append(f"{p.name}: {p.N}^2 grid, {p.s}x{p.s} subdomains")
    setup = time.perf_counter() - t0
    solve_batch(solvers, max(3, args.warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solve_batch(solvers, args.steps)
    wall = time.perf_counter() - t0
    ms = st[0]["ms"]
    dofs = sum((p.N - 1) ** 2 * p.P for p in probs)
    line = {"metric": "batched SG-DD problem-steps/sec (uneven problems, one graph launch per step)",
            "value": len(probs) * args.steps / (ms / 1e3), "unit": "problem-steps/s", "problems": len(probs),
            "steps": args.steps, "ms_per_batch_step": ms / args.steps, "wall_s": wall, "setup_s": setup,
            "total_sg_dofs": dofs, "pcg_iters_per_step": sum(s["iters_total"] for s in st) / (len(st) * args.steps),
            "max_iters_last": max(s["iters_last"] for s in st), "dtype": "f32+f64", "data": "synthetic",
            "skipped": skipped, "warm_start": args.batch_warm,
            "config": {"workload": "batch (seed 20251227)", "grids": sorted({p.N for p in probs}),
                       "subdomains": sorted({p.s for p in probs}), "pce_terms": sorted({p.P for p in probs})}}
    print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()
    return 0


def ricker_nodal_load(prob, step_from, nsteps, nf):
    """Host copy of the workload's deterministic load: the Ricker point source's P1 nodal values for
    steps step_from + 1 .. step_from + nsteps (the user's input of the end-to-end leg)."""
    import numpy as np
    src0 = prob.source
    N, h = prob.N, 1.0 / prob.N
    i = min(int(math.floor(src0.x0 / h)), N - 1)
    j = min(int(math.floor(src0.y0 / h)), N - 1)
    fx, fy = src0.x0 / h - i, src0.y0 / h - j
    if fy <= fx:
        nodes = [((i, j), 1 - fx), ((i + 1, j), fx - fy), ((i + 1, j + 1), fy)]
    else:
        nodes = [((i, j), 1 - fy), ((i + 1, j + 1), fx), ((i, j + 1), fy - fx)]
    fidx = [((b - 1) * (N - 1) + (a - 1), v) for (a, b), v in nodes if 1 <= a <= N - 1 and 1 <= b <= N - 1 and v]
    out = np.zeros((nsteps, nf))
    for k in range(nsteps):
        t = (step_from + k + 1) * prob.dt
        tau = t - 1.0 / src0.freq
        a2 = (math.pi * src0.freq * tau) ** 2
        r = src0.amp * (1 - 2 * a2) * math.exp(-a2)
        for fi, v in fidx:
            out[k, fi] = r * v
    return out


def run_precond_study(args):
    """Comparison of the interface preconditioners (the paper's Sec. 6.1 experiment on structured
    grids): a fixed 256^2 grid (the 1024^2 workload's field and PCE sizes: M = 5, order 2, sigma 0.3,
    correlation length 0.1, Ricker source) split into s x s subdomains, s = 2, 4, 8, 16; for the
    two-level Neumann-Neumann preconditioner of the method, the one-level Neumann-Neumann and the
    lumped one: average outer PCG iterations per step and ms per step over `steps` steps (mixed
    precision, tolerance 1e-8), after `warmup` steps."""
    import sg_workloads as w
    from paper_2512_23027_gb300 import Solver
    from paper_2512_23027_gb300.binding import SG_MIXED
    if args.mesh:
        return run_precond_study_mesh(args)
    base = w.config("ricker1024").replace(name="pc256", N=256, dt=w.cfl_dt(256))
    rows = []
    for s in (2, 4, 8, 16):
        for name, pc in (("two-level NN", 0), ("one-level NN", 1), ("lumped", 2)):
            prob = base.replace(s=s)
            sv = Solver(prob, precision=SG_MIXED, precond=pc)
            sv.step(args.warmup)
            st = sv.step(args.steps)
            rows.append({"subdomains": f"{s}x{s}", "precond": name, "outer_iters_per_step": st["iters_total"] / args.steps,
                         "inner_iters_per_step": st["inner_total"] / args.steps, "ms_per_step": st["ms"] / args.steps})
            sv.close()
    print(json.dumps({"metric": "outer PCG iterations per step vs number of subdomains, by preconditioner",
                      "config": {"workload": "256x256 grid, M=5, order 2 (P=21), sigma 0.3, corr 0.1, Ricker, "
                                             "mixed precision, tol 1e-8", "warmup": args.warmup, "steps": args.steps},
                      "rows": rows}), flush=True)
    return 0


def run_mesh(args):
    """Mesh workload (a seeded unstructured mesh with an RCB partition, sg_setup_mesh): steps/s of the
    mixed solver with the learned warm start and of the plain FP64 solver with the previous-step guess,
    on the same GPU, from the same initial state; `warmup` untimed steps each, then one sg_step per
    timed step (CUDA events on the solver's stream) with a 256 MB buffer written between steps."""
    import torch
    import sg_workloads as w
    from paper_2512_23027_gb300 import Solver
    from paper_2512_23027_gb300.binding import SG_BF16, SG_FP64, SG_MIXED, SG_WARM_LEARNED, SG_WARM_PREV
    c = w.mesh_config(args.mesh)
    mesh = c.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    legs = {}
    plan = [("mixed_learned", SG_MIXED, SG_WARM_LEARNED, args.steps),
            ("fp64", SG_FP64, SG_WARM_PREV, min(args.steps, args.fp64_steps))]
    if c.prob.P <= 32:   # the tensor-core mean-operator product (SG_BF16) where it applies
        plan.insert(1, ("bf16_learned", SG_BF16, SG_WARM_LEARNED, args.steps))
    for key, precision, warm, K in plan:
        t0 = time.perf_counter()
        sv = Solver(c.prob, precision=precision, warm=warm, stream=stream, mesh=mesh)
        setup = time.perf_counter() - t0
        sv.step(max(3, args.warmup))
        ms, outer, inner = 0.0, 0, 0
        for k in range(K):
            flush.fill_(float(k))
            st = sv.step(1)
            ms += st["ms"]
            outer += st["iters_total"]
            inner += st["inner_total"]
        legs[key] = {"steps_per_s": K / (ms / 1e3), "ms_per_step": ms / K, "outer_iters_per_step": outer / K,
                     "inner_iters_per_step": inner / K, "steps": K, "setup_s": setup,
                     "device_bytes": sv.sizes["device_bytes"]}
        if key != "fp64":
            # per-kernel CUDA-event times of one host-driven step each: class 1 the preconditioner product
            # of the subdomain CG, class 2 its operator apply (untimed for the line above)
            sv.set_eager(True)
            sv.kernel_timing(1)
            sv.step(1)
            ms1, n1 = sv.kernel_timing(2)
            sv.step(1)
            ms2, n2 = sv.kernel_timing(0)
            sv.set_eager(False)
            legs[key]["kernels"] = {"precond_product": {"avg_launch_us": 1e3 * ms1 / n1 if n1 else None, "launches": n1},
                                    "inner_apply": {"avg_launch_us": 1e3 * ms2 / n2 if n2 else None, "launches": n2}}
        sv.close()
    p = c.prob
    line = {"metric": "time-steps/sec on a general partition of an unstructured mesh (mixed precision + learned "
                      "warm start; plain FP64 beside it)",
            "value": legs["mixed_learned"]["steps_per_s"], "unit": "steps/s", "higher_is_better": True,
            "steps": args.steps, "warmup": max(3, args.warmup), "dtype": "f32+f64", "data": "synthetic",
            "speedup_vs_fp64": legs["mixed_learned"]["steps_per_s"] / legs["fp64"]["steps_per_s"],
            "mixed_learned": legs["mixed_learned"], "fp64": legs["fp64"], "bf16_learned": legs.get("bf16_learned"),
            "config": {"workload": c.name, "vertices": int(mesh[0].shape[0]), "triangles": int(mesh[2].shape[0]),
                       "subdomains": c.nparts, "M": p.M, "p": p.p, "P": p.P, "dt": p.dt, "tol": p.tol,
                       "l2": "256 MB buffer written between timed steps"}}
    print(json.dumps(line), flush=True)
    return 0


def run_precond_study_mesh(args):
    """The preconditioner comparison on a mesh workload (--mesh NAME; umesh_e1 is the paper's Sec. 6.1
    setting: a 1600-vertex unstructured mesh, deterministic medium, dt 0.01): RCB partitions into 2 .. 64
    subdomains, the two-level NN, one-level NN and lumped preconditioners, mixed precision, tolerance
    1e-8; average outer PCG iterations and ms per step over `steps` steps after `warmup` steps."""
    import sg_workloads as w
    from sg_workloads import meshes
    from paper_2512_23027_gb300 import Solver
    from paper_2512_23027_gb300.binding import SG_MIXED
    c = w.mesh_config(args.mesh)
    xy, d, tri, _ = c.build()
    rows = []
    for nparts in (2, 4, 8, 16, 32, 64):
        part = meshes.rcb_partition(xy, tri, nparts)
        for name, pc in (("two-level NN", 0), ("one-level NN", 1), ("lumped", 2)):
            sv = Solver(c.prob, precision=SG_MIXED, precond=pc, mesh=(xy, d, tri, part))
            sv.step(args.warmup)
            st = sv.step(args.steps)
            rows.append({"subdomains": nparts, "precond": name, "outer_iters_per_step": st["iters_total"] / args.steps,
                         "inner_iters_per_step": st["inner_total"] / args.steps, "ms_per_step": st["ms"] / args.steps})
            sv.close()
    print(json.dumps({"metric": "outer PCG iterations per step vs number of subdomains, by preconditioner (mesh)",
                      "config": {"workload": c.name, "vertices": int(xy.shape[0]), "M": c.prob.M, "P": c.prob.P,
                                 "dt": c.prob.dt, "precision": "mixed", "tol": c.prob.tol, "warmup": args.warmup,
                                 "steps": args.steps}, "rows": rows}), flush=True)
    return 0


def run_profile_step(args):
    """One step of the workload for profilers (mixed precision, learned warm start; with --profile-fp64
    the plain FP64 solver): fast-forward (graph mode), one untimed host-driven step,
    then one host-driven step between cudaProfilerStart / cudaProfilerStop (run ncu with
    --profile-from-start off).  Host-driven enqueue launches the same kernels as the step graph, which
    per-kernel profilers cannot enter (conditional nodes)."""
    import torch
    import sg_workloads as w
    from paper_2512_23027_gb300 import Solver
    from paper_2512_23027_gb300.binding import SG_FP64, SG_MIXED, SG_WARM_LEARNED
    if args.mesh:   # a mesh workload (--mesh NAME): its mixed solver with the learned warm start
        c = w.mesh_config(args.mesh)
        prob, mesh = c.prob, c.build()
        F = 20 if args.forward is None else args.forward
    else:
        prob, mesh = w.config(args.config), None
        F = FORWARD.get(args.config, 0) if args.forward is None else args.forward
    s = Solver(prob, precision=SG_MIXED, warm=SG_WARM_LEARNED, mesh=mesh)   # the benchmark's optimised configuration
    if F:
        s.step(F)
    if args.profile_fp64:
        st0 = s.get_state()
        s.close()
        s = Solver(prob, precision=SG_FP64, mesh=mesh)
        s.set_state(st0)
    s.set_eager(True)
    s.step(1)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    st = s.step(1)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profiled_step": st["step_index"], "iters": st["iters_total"], "inner": st["inner_total"]}))
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="ricker1024")
    ap.add_argument("--forward", type=int, default=None,
                    help="untimed steps before the warm-up (default: the workload's, 200 at 1024^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the default line, run the first BATCH problems of the batched workload "
                         "(64^2..256^2 grids, uneven sizes) with sg_solve_batch and report problem-steps/s")
    ap.add_argument("--batch-warm", default="learned", choices=["learned", "prev"],
                    help="with --batch: the PCG initial guess of every problem")
    ap.add_argument("--precond-study", action="store_true",
                    help="instead of the default line, compare the two-level NN, one-level NN and lumped "
                         "preconditioners over 2x2..16x16 subdomains of a 256^2 grid (iterations per step)")
    ap.add_argument("--profile-step", action="store_true",
                    help="instead of the default line: fast-forward, then one host-driven step between "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--profile-fp64", action="store_true", help="with --profile-step: the plain FP64 solver")
    ap.add_argument("--mesh", default=None,
                    help="time a mesh workload instead (umesh_small, umesh13k, umesh37k, umesh37k_rv9, umesh37k_720, "
                         "umesh_e1): a seeded unstructured mesh with an RCB partition, mixed + learned warm start, "
                         "SG_BF16 where P <= 32, and plain FP64; with --precond-study the preconditioner comparison "
                         "on that mesh, with --profile-step one host-driven step of it")
    ap.add_argument("--enqueue", default="graph", choices=["graph", "eager"],
                    help="graph: one CUDA graph per step (default); eager: host-driven enqueue of the same "
                         "kernels (per-kernel profilers cannot see inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    if args.precond_study:
        return run_precond_study(args)   # with --mesh NAME: on that mesh
    if args.profile_step:
        return run_profile_step(args)   # with --mesh NAME: a step of that mesh workload
    if args.mesh:
        return run_mesh(args)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    # the CPU baseline processes start before this process touches the GPU
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc = start_cpu_baseline(args.config, args.cpu_steps)

    import torch
    import sg_workloads as w
    from paper_2512_23027_gb300 import Solver
    from paper_2512_23027_gb300.binding import SG_FP64, SG_MIXED, SG_WARM_LEARNED, SG_WARM_PREV

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    prob = w.config(args.config)
    K, W = args.steps, max(args.warmup, 3)
    F = FORWARD.get(args.config, 0) if args.forward is None else args.forward
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(solver, nsteps):
        its, inner, ms = [], 0, 0.0
        for k in range(nsteps):
            flush.fill_(float(k))
            st = solver.step(1)
            ms += st["ms"]
            its.append(st["iters_total"])
            inner += st["inner_total"]
        return ms, its, inner

    eager = args.enqueue == "eager"

    def make(p, precision, warm=SG_WARM_PREV):
        sv = Solver(p, precision=precision, stream=stream, warm=warm)
        if eager:
            sv.set_eager(True)
        return sv

    # ---- optimised solver (mixed precision, learned warm start, graph per step): fast-forward,
    # warm-up, timed steps ----
    t_setup = time.perf_counter()
    s = make(prob, SG_MIXED, SG_WARM_LEARNED)
    t_setup = time.perf_counter() - t_setup
    t_fwd = time.perf_counter()
    if F:
        s.step(F)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t_fwd
    state0 = s.get_state()            # step F: the state every leg starts from
    s.step(W)
    sampler = ClockSampler(bus_id_of(torch, local))
    barrier()
    l0 = s.launch_count()
    sampler.start()
    torch.cuda.nvtx.range_push("timed")
    ms, its, inner = timed(s, K)
    torch.cuda.nvtx.range_pop()
    barrier()
    clocks = sampler.stop()
    launches = s.launch_count() - l0
    tmax = max_over_ranks(ms, dist, "cuda")
    value = world * K / (tmax / 1e3)

    # ---- dominant kernel: CUDA-event timing of each of its launches (host-driven enqueue) ----
    tc = s.sizes.get("fp32_precond", 0) == 1
    s.set_eager(True)
    s.kernel_timing(3 if tc else 1)
    kr = min(K, 3)
    for k in range(kr):
        flush.fill_(float(k))
        s.step(1)
    kms, kn = s.kernel_timing(0)
    s.kernel_timing(2)
    for k in range(kr):
        flush.fill_(float(k))
        s.step(1)
    ams, an = s.kernel_timing(0)
    s.kernel_timing(4)
    for k in range(kr):
        flush.fill_(float(k))
        s.step(1)
    oms, on = s.kernel_timing(0)
    s.set_eager(eager)
    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs")
    kbytes = tc_product_bytes(prob) if tc else line_kernel_bytes(prob, 4)
    kdur = (kms / kn / 1e3) if kn else None
    achieved = kbytes / kdur / 1e9 if kdur else None
    ksha = kernel_source_sha()
    kname = ("k_pre_mma<32> (BF16 dense inverse of the mean operator x [r_hi; r_lo] on tcgen05, TMA-fed, "
             "FP32 accumulation in TMEM)" if tc else
             "k_line_w<float> (register-tiled FP32 mean-operator line sweeps fused with the inner CG update)")
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if (achieved and hbm) else None, "traffic": KERNEL_TRAFFIC.get(ksha),
                "launches_timed": kn, "avg_launch_us": 1e3 * kms / kn if kn else None,
                "bytes_per_launch": kbytes, "peak_source": "measured" if hbm else "fallback",
                "source_sha": ksha,
                "bytes_note": "method bytes: 7 inner-CG vector passes + the L^3 line factor of every subdomain "
                              "(FP32), all subdomain problems active (timed after the fast-forward)",
                "apply_kernel": {"avg_launch_us": 1e3 * ams / an if an else None, "launches_timed": an},
                "outer_apply_kernel": {"avg_launch_us": 1e3 * oms / on if on else None, "launches_timed": on,
                                       "what": "operator applies with FP64 inputs and outputs (effective load, "
                                               "residual corrections)"}}
    if tc and kdur:
        bf16 = peaks.get("bf16_tflops")
        tfl = tc_product_flops(prob) / kdur / 1e12
        roofline["tensor"] = {"achieved": tfl, "peak": bf16, "unit": "TFLOP/s",
                              "frac": tfl / bf16 if bf16 else None, "flops_per_launch": tc_product_flops(prob)}
    if not hbm:
        roofline["peak"] = 6800.0
        roofline["frac"] = achieved / 6800.0 if achieved else None
        roofline["peak_source"] = "fallback"

    # ---- end to end through the C ABI with pinned host buffers, from the same state ----
    pe = prob.replace(source=w.Source())
    se = make(pe, SG_MIXED, SG_WARM_LEARNED)
    se.set_state(state0)
    se.warm_weights(s.warm_weights())   # the network the optimised leg trained (no retraining)
    nf = se.n_free
    fw = torch.from_numpy(ricker_nodal_load(prob, F, W, nf)).pin_memory()
    uw = torch.zeros((W, nf), dtype=torch.float64).pin_memory()
    fh = torch.zeros((K, nf), dtype=torch.float64).pin_memory()
    uh = torch.zeros((K, nf), dtype=torch.float64).pin_memory()
    se.step_host(W, fw, uw)
    fh.numpy()[:] = ricker_nodal_load(prob, F + W, K, nf)   # the user's inputs, resident in pinned host memory
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_e = se.step_host(K, fh, uh)     # per step: H2D of the load, the step, D2H of the mean field
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": world * K / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": nf * 8,
           "d2h_bytes_per_step": nf * 8, "pcg_iters_per_step": st_e.get("iters_total", 0) / K,
           "note": "sg_step_host from the fast-forwarded state (host clock around the call): per step H2D of "
                   "the nodal load from pinned host memory, one SG-DD step, D2H of the mean field into pinned "
                   "host memory"}
    se.close()
    s.close()

    # ---- plain FP64 DD-PCG on the same GPU, from the same state ----
    s64 = make(prob, SG_FP64)
    s64.set_state(state0)
    s64.step(1)
    barrier()
    K64 = max(1, min(args.fp64_steps, K))
    ms64, its64, inner64 = timed(s64, K64)
    barrier()
    ms64 = max_over_ranks(ms64, dist, "cuda")
    s64.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = finish_cpu_baseline(cpu_proc, args.config, args.cpu_steps, timeout=900)
    cfg = workload_config(prob, "mixed (fp32 subdomain, fp64 outer)")
    cfg["warm_start"] = ("learned: Newmark predictor + least-squares autoregressive model of its error, refitted "
                         "every step, + gated network correction (plain FP64 arm: previous-step solution)")
    cfg["window"] = (f"steps {F + W + 1}..{F + W + K} of the run: {F} untimed fast-forward steps and {W} warm-up "
                     f"steps first" if F else f"steps {W + 1}..{W + K}")
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "config": cfg,
            "pcg_iters_per_step": sum(its) / K, "inner_iters_per_step": inner / K,
            "plain_fp64": {"value": world * K64 / (ms64 / 1e3), "unit": "steps/s", "ms_per_step": ms64 / K64,
                           "pcg_iters_per_step": sum(its64) / K64, "inner_iters_per_step": inner64 / K64,
                           "steps": K64},
            "speedup_vs_plain_fp64": (value / (world * K64 / (ms64 / 1e3))),
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": launches, "enqueue": args.enqueue,
            "setup_s": t_setup, "forward_s": t_fwd, "forward_steps": F}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
