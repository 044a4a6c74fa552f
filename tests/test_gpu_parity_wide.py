"""GPU parity on subdomains of 65 x 65 and 121 x 121 nodes (the register-tiled line sweeps of both
precisions, the compiled triple-product tables of the 512^2 and 1024^2 workloads) against stored
samples of the CPU oracle's DD-PCG (tests/golden/oracle_samples.json, written by
tests/golden/make_oracle_samples.py, which calls only the oracle).

Each case is advanced the oracle's number of steps at the oracle's PCG tolerance: 1e-13 for the FP64
path, the workload tolerance 1e-8 for mixed precision.  Compared: the values of U at the stored
(free node, mode) entries, the l2 norm of every PCE mode of U over all free nodes, and the outer
iteration counts.  The entries are n_uniform uniform draws and the oracle's largest-magnitude
entries (where the wave is).  On the uniform draws, RMS(U - U_ref) / (||U_ref|| / sqrt(n_free P))
estimates ||U - U_ref|| / ||U_ref||, and per mode k RMS_k(U - U_ref) / (max(||U_ref,k||, 1e-3 ||U_ref||)
/ sqrt(n_free)) estimates ||U_k - U_ref,k|| / ||U_ref,k|| (modes smaller than 1e-3 of the field against
1e-3 of it).  On the largest entries the relative l2 error over those entries is reported."""
import json
import os

import numpy as np
import pytest

import sg_workloads as w

pytestmark = pytest.mark.gpu

GOLD_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_samples.json")
SG_FP64, SG_MIXED, SG_BF16 = 0, 1, 3


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    return Solver


def gold():
    return json.load(open(GOLD_PATH))


def problem(name, rec):
    p, s = rec["problem"], rec["source"]
    return w.Problem(name, N=p["N"], s=p["s"], M=p["M"], p=p["p"], p_in=p["p_in"], sigma=p["sigma"], bx=p["bx"],
                     by=p["by"], g0=p["g0"], dt=p["dt"], steps=rec["steps"], tol=p["tol"],
                     source=w.Source(**s), alpha0=p["alpha0"], alpha1=p["alpha1"])


def compare(U, rec, ref):
    node, mode = np.array(rec["node"]), np.array(rec["mode"])
    vals = np.array(ref["values"])
    mnorm = np.array(ref["mode_norm"])
    nu = rec.get("n_uniform", node.size)
    nf = U.shape[0]
    d = U[node, mode] - vals
    du, mu = d[:nu], mode[:nu]
    glob = np.sqrt(np.mean(du ** 2)) / (ref["norm"] / np.sqrt(nf * U.shape[1]))
    per_mode = []
    floor = 1e-3 * ref["norm"]
    for k in range(U.shape[1]):
        sel = mu == k
        per_mode.append(np.sqrt(np.mean(du[sel] ** 2)) / (max(mnorm[k], floor) / np.sqrt(nf)) if sel.any() else 0.0)
    norm_rel = np.abs(np.linalg.norm(U, axis=0) - mnorm) / np.maximum(mnorm, floor)
    top = np.linalg.norm(d[nu:]) / np.linalg.norm(vals[nu:]) if nu < node.size else 0.0
    return glob, np.array(per_mode), norm_rel, top


# Stated bars (sampled estimates of relative l2 errors).  FP64 at PCG tolerance 1e-13: 1e-10 for the
# field, 1e-9 per mode.  Mixed precision at the workload tolerance tol = 1e-8, the error model of the
# small-problem tests: both solvers stop at ||r|| <= tol ||G||, so 10 tol for the field (the error of
# the whole field), and a mode holds at most all of it: 10 tol ||U|| / ||U_k|| <= 1e4 tol per mode
# with the 1e-3 floor.
BARS = {SG_FP64: {"glob": 1e-10, "mode": 1e-9}, SG_MIXED: {"glob": 1e-7, "mode": 1e-4},
        SG_BF16: {"glob": 1e-7, "mode": 1e-4}}


@pytest.mark.slow
@pytest.mark.parametrize("precision", [SG_FP64, SG_MIXED, SG_BF16], ids=["fp64", "mixed", "bf16"])
@pytest.mark.parametrize("case", ["l65_m5p2", "l65_m4p3", "b240"])
def test_wide_subdomains_match_oracle_samples(lib, case, precision):
    """SG_BF16 runs the line sweeps with their per-line products on the tensor cores (65 x 65-node
    subdomains; the 121 x 121-node case has no BF16 preconditioner and is skipped)."""
    g = gold()
    if case not in g:
        pytest.skip(f"{case} not in the stored oracle samples")
    if precision == SG_BF16 and case == "b240":
        pytest.skip("no BF16 tensor-core preconditioner for 121 x 121-node subdomains")
    rec = g[case]
    prob = problem(case, rec)
    ref = rec["tight"] if precision == SG_FP64 else rec["workload"]
    s = lib(prob, precision=precision, tol=ref["tol"])
    plan_line = s.sizes
    s.step(rec["steps"])
    U = s.field()
    its, rr = s.iters()
    s.close()
    glob, per_mode, norm_rel, top = compare(U, rec, ref)
    print(f"{case} {({SG_FP64: 'fp64', SG_MIXED: 'mixed', SG_BF16: 'bf16'})[precision]}: sampled rel err {glob:.3e}, largest entries "
          f"{top:.3e}, worst mode {per_mode.max():.3e} (mode {int(per_mode.argmax())}), mode-norm rel diff "
          f"{norm_rel.max():.3e}, iters {its} vs {ref['iters']}, {plan_line['P']} modes")
    bar = BARS[precision]
    assert glob <= bar["glob"], glob
    assert top <= bar["glob"], top
    assert per_mode.max() <= bar["mode"], per_mode
    assert norm_rel.max() <= bar["mode"], norm_rel
    assert all(r <= ref["tol"] for r in rr)
    assert all(abs(a - b) <= 1 for a, b in zip(its, ref["iters"]))


@pytest.mark.slow
@pytest.mark.parametrize("case", ["l65_m5p2", "l65_m4p3"])
def test_learned_warm_start_on_wide_subdomains(lib, case):
    """The benchmark's configuration (mixed precision with the learned warm start) on 65 x 65-node
    subdomains against the stored oracle samples (previous-step guess, workload tolerance): the warm
    start changes the PCG's starting point only, so the mixed-precision bars hold."""
    from paper_2512_23027_gb300.binding import SG_WARM_LEARNED
    g = gold()
    if case not in g:
        pytest.skip(f"{case} not in the stored oracle samples")
    rec = g[case]
    prob = problem(case, rec)
    ref = rec["workload"]
    s = lib(prob, precision=SG_MIXED, tol=ref["tol"], warm=SG_WARM_LEARNED)
    s.step(rec["steps"])
    U = s.field()
    its, rr = s.iters()
    s.close()
    glob, per_mode, norm_rel, top = compare(U, rec, ref)
    print(f"{case} mixed + learned warm start: sampled rel err {glob:.3e}, largest entries {top:.3e}, worst mode "
          f"{per_mode.max():.3e}, iters {its} vs {ref['iters']}")
    bar = BARS[SG_MIXED]
    assert glob <= bar["glob"] and top <= bar["glob"]
    assert per_mode.max() <= bar["mode"] and norm_rel.max() <= bar["mode"]
    assert all(r <= ref["tol"] for r in rr)
