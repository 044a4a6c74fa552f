"""GPU parity: the CUDA SG-DD path against the FP64 CPU oracle (same inputs, element by
element over every free node and PCE mode).  Bar: relative l2 error <= 1e-10 in FP64 mode
with PCG tolerance 1e-13 on both sides; iteration counts at the workload tolerance equal to
the oracle's within one."""
import numpy as np
import pytest

import sg_workloads as w
from oracle import dd as odd, sg as osg

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    return Solver


def oracle_run(prob, steps, tol):
    sgp = osg.SGProblem(prob)
    d = odd.DDSolver(prob)
    U, V, A, it = odd.run_dd(sgp, d, steps, tol=tol)
    return U.reshape(-1, prob.P), V.reshape(-1, prob.P), A.reshape(-1, prob.P), [i for i, _ in it]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rel_modes(a, b, floor=1e-3):
    """||a_k - b_k|| / max(||b_k||, floor ||b||) for every PCE mode k (columns): each mode against its
    own norm, except modes smaller than `floor` of the whole field (in early steps the highest modes
    can be 1e-6 of the mean), which are measured against floor ||b||."""
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), floor * np.linalg.norm(b))


# Bars of the FP64 path at PCG tolerance 1e-13 on both sides.  U: 1e-10 relative over all nodes and
# modes, 1e-9 for every mode on its own (the higher modes are orders of magnitude smaller than the
# mean).  V and A come from U through the Newmark relations: a_{n+1} = u_{n+1} / (zeta dt^2) - u~_m
# subtracts two terms each about 1 / (omega dt)^2 times larger than a_{n+1} itself, so U's relative
# error reaches A amplified by that factor (dt = 0.02 on the 8^2 problem: about 10^2) and V through
# the trapezoidal update by about half of it.
BAR_U, BAR_U_MODE, BAR_V, BAR_A = 1e-10, 1e-9, 1e-9, 1e-8


@pytest.mark.parametrize("name,steps", [("tiny", 5), ("small", 4), ("pulse32", 5)])
def test_fp64_matches_oracle(lib, name, steps):
    prob = w.config(name)
    s = lib(prob, tol=1e-13)
    st = s.step(steps)
    U = s.field()
    state = s.get_state()
    s.close()
    Ur, Vr, Ar, _ = oracle_run(prob, steps, 1e-13)
    n = prob.P * Ur.shape[0]
    V = state[n:2 * n].reshape(Vr.shape)
    A = state[2 * n:3 * n].reshape(Ar.shape)
    print(f"{name}: U {rel(U, Ur):.2e} (worst mode {rel_modes(U, Ur).max():.2e}), V {rel(V, Vr):.2e}, "
          f"A {rel(A, Ar):.2e}")
    assert rel(U, Ur) <= BAR_U, rel(U, Ur)
    assert rel_modes(U, Ur).max() <= BAR_U_MODE, rel_modes(U, Ur)
    assert rel(V, Vr) <= BAR_V
    assert rel(A, Ar) <= BAR_A
    assert st["step_index"] == steps


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_input_order_twice_output_order(lib, precision):
    """p_in = 2 p: the log-normal coefficient expanded to order 4 with the solution at order 2 (the
    projection of the truncated field is then exact), runtime triple-product table (no compiled
    table for p_in != p), against the oracle at the same tolerance."""
    prob = w.config("small").replace(name="pin4", p_in=4)
    tol = 1e-13 if precision == 0 else 1e-10
    steps = 3
    s = lib(prob, precision=precision, tol=tol)
    assert s.sizes["P_in"] == 15 and s.sizes["compiled_apply"] == 0
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    Ur, _, _, its_ref = oracle_run(prob, steps, tol)
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"p_in = 4, p = 2, {'fp64' if precision == 0 else 'mixed'}: rel err {err:.2e}, worst mode {modes:.2e}, "
          f"iters {its} vs {its_ref}")
    if precision == 0:
        assert err <= BAR_U and modes <= BAR_U_MODE
    else:
        assert err <= BAR_MIXED * tol and modes <= BAR_MIXED_MODE * tol
    assert all(r <= tol for r in rr)
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_ref))


@pytest.mark.parametrize("name", ["small", "pulse32"])
def test_iteration_counts_match_oracle(lib, name):
    prob = w.config(name)
    steps = 4
    s = lib(prob)
    s.step(steps)
    its, rr = s.iters()
    s.close()
    _, _, _, its_ref = oracle_run(prob, steps, prob.tol)
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_ref)), (its, its_ref)
    assert all(r <= prob.tol for r in rr)


def test_checkpoint_resume_bitwise(lib):
    prob = w.config("small")
    a = lib(prob)
    a.step(2)
    st = a.get_state()
    a.step(2)
    ua = a.field()
    b = lib(prob)
    b.set_state(st)
    b.step(2)
    ub = b.field()
    assert np.array_equal(ua, ub)
    a.close(); b.close()


def test_moments(lib):
    prob = w.config("small")
    s = lib(prob)
    s.step(3)
    U = s.field()
    m, v = s.moments()
    assert np.array_equal(m, U[:, 0])
    assert np.allclose(v, np.sum(U[:, 1:] ** 2, axis=1), rtol=1e-14, atol=0)
    s.close()


# Mixed precision: FP32 subdomain solves with one FP64 residual correction per Dirichlet solve
# inside an FP64 outer PCG.  Both sides stop at ||r|| <= tol ||G||, so the fields differ by the
# error both solvers leave at that residual: the bar is 10 tol relative over all nodes and modes
# (measured 0.4 - 3 tol).  That bound holds for the whole field; a mode k holds at most all of it, so
# its own relative error is bounded by 10 tol ||U|| / ||U_k||, at most 1e4 tol with the 1e-3 floor of
# rel_modes (measured up to 2.1e3 tol on the 5-step pulse, whose second mode is 3e-3 of the field).
BAR_MIXED, BAR_MIXED_MODE = 10.0, 1e4


@pytest.mark.parametrize("name,steps", [("small", 4), ("pulse32", 5)])
def test_mixed_matches_oracle(lib, name, steps):
    from paper_2512_23027_gb300.binding import SG_MIXED
    prob = w.config(name)
    s = lib(prob, precision=SG_MIXED)
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    Ur, _, _, its_ref = oracle_run(prob, steps, prob.tol)
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"{name}: mixed vs oracle rel err {err:.3e} ({err / prob.tol:.2f} tol), worst mode {modes:.3e}, "
          f"iters {its} vs {its_ref}")
    assert err <= BAR_MIXED * prob.tol, err
    assert modes <= BAR_MIXED_MODE * prob.tol, modes
    assert all(r <= prob.tol for r in rr)
    assert all(a <= b + 2 for a, b in zip(its, its_ref))


@pytest.mark.parametrize("name,steps", [("small", 4), ("pulse32", 5)])
def test_float_float_outer_applies(lib, name, steps):
    """The operator applies of the mixed path's FP64 outer loop (effective load, residual corrections)
    run in float-float pairs where the compiled triple-product table applies, about 1e-13 relative;
    SG_APPLY_FP64 runs them in FP64.  Both give the same outer iteration counts within one and fields
    within the solver tolerance of each other, each within the mixed-precision bar of the oracle."""
    from paper_2512_23027_gb300.binding import SG_MIXED
    prob = w.config(name)
    ua, ia, ra = _run_env(lib, prob, SG_MIXED, steps, {})
    ub, ib, rb = _run_env(lib, prob, SG_MIXED, steps, {"SG_APPLY_FP64": "1"})
    Ur, _, _, _ = oracle_run(prob, steps, prob.tol)
    print(f"{name}: float-float vs FP64 outer applies rel diff {rel(ua, ub):.3e}, vs oracle {rel(ua, Ur):.3e} / "
          f"{rel(ub, Ur):.3e}, iters {ia} vs {ib}")
    assert rel(ua, ub) <= prob.tol
    assert rel(ua, Ur) <= BAR_MIXED * prob.tol and rel(ub, Ur) <= BAR_MIXED * prob.tol
    assert all(r <= prob.tol for r in ra + rb)
    assert all(abs(x - y) <= 1 for x, y in zip(ia, ib))


def test_graph_equals_eager(lib):
    """The captured step graph (conditional WHILE/IF nodes) and the host-driven enqueue of
    the same kernels give bitwise identical results."""
    import os
    prob = w.config("small")
    a = lib(prob)
    a.step(3)
    ua = a.field()
    a.close()
    os.environ["SG_EAGER"] = "1"
    try:
        b = lib(prob)
        b.step(3)
        ub = b.field()
        b.close()
    finally:
        del os.environ["SG_EAGER"]
    assert np.array_equal(ua, ub)


def test_tensor_core_preconditioner_matches_line_sweeps(lib):
    """Mixed precision on the 128^2 / P = 20 workload: the FP32 subdomain CG preconditioned by the
    dense BF16 inverse of the mean operator on the tensor cores (with the compiled triple-product
    apply) and by the exact line sweeps (runtime-table apply) converge to the same fields.  Both runs
    stop at the outer tolerance, so they agree to a small multiple of it; outer iteration counts
    agree within one."""
    import os
    from paper_2512_23027_gb300.binding import SG_MIXED
    prob = w.config("ricker128")
    steps = 6
    a = lib(prob, precision=SG_MIXED)
    assert a.sizes["fp32_precond"] == 1 and a.sizes["compiled_apply"] == 1
    a.step(steps)
    ua, (ia, ra) = a.field(), a.iters()
    a.close()
    os.environ["SG_NO_MMA"] = "1"
    os.environ["SG_NO_GFIX"] = "1"
    try:
        b = lib(prob, precision=SG_MIXED)
        assert b.sizes["fp32_precond"] == 0 and b.sizes["compiled_apply"] == 0
        b.step(steps)
        ub, (ib, rb) = b.field(), b.iters()
        b.close()
    finally:
        del os.environ["SG_NO_MMA"]
        del os.environ["SG_NO_GFIX"]
    err = rel(ua, ub)
    print(f"tensor-core vs line-sweep preconditioner: rel diff {err:.3e}, iters {ia} vs {ib}")
    assert err <= 1e2 * prob.tol, err
    assert all(r <= prob.tol for r in ra) and all(r <= prob.tol for r in rb)
    assert all(abs(x - y) <= 1 for x, y in zip(ia, ib))


@pytest.mark.parametrize("N,M,p", [(38, 4, 2), (22, 3, 2), (24, 3, 3)])
def test_tensor_core_preconditioner_empty_trailing_chunk(lib, N, M, p):
    """Subdomain sizes whose L^2 nodes leave the last 64-node chunk of the 128-padded rows of the
    dense inverse empty (L = 20, 12, 13) with nl * P a multiple of four, so that the residual image
    is packed with 16-byte vectors: P = 15 and 10 (16 image rows) and P = 20 (32 rows).  Mixed
    precision with the tensor-core preconditioner against the oracle's DD-PCG at the same
    tolerance."""
    from paper_2512_23027_gb300.binding import SG_MIXED
    base = w.config("ricker128")
    prob = base.replace(name=f"chunk{N}", N=N, s=2, M=M, p=p, p_in=p, dt=w.cfl_dt(N))
    L = N // 2 + 1
    assert (L * L) % 128 <= 64 and (L * L * prob.P) % 4 == 0
    steps = 4
    s = lib(prob, precision=SG_MIXED)
    assert s.sizes["fp32_precond"] == 1
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    Ur, _, _, its_ref = oracle_run(prob, steps, prob.tol)
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"L={L} P={prob.P}: tensor-core mixed vs oracle rel err {err:.3e}, worst mode {modes:.3e}, "
          f"iters {its} vs {its_ref}")
    assert err <= BAR_MIXED * prob.tol, err
    assert modes <= BAR_MIXED_MODE * prob.tol, modes
    assert all(r <= prob.tol for r in rr)
    assert all(a <= b + 2 for a, b in zip(its, its_ref))


@pytest.mark.slow
def test_bench_workload_mixed_matches_oracle(lib):
    """The timed workload itself (128^2 grid, 4 x 4 subdomains, P = 20, workload tolerance 1e-8) in
    the configuration bench.py times (mixed precision, tensor-core preconditioner, CUDA graph), two
    steps against the oracle's DD-PCG at the same tolerance.  Both stop at ||r|| / ||G|| <= 1e-8, so
    the fields agree to a small multiple of it; every step converges and the outer iteration counts
    agree within one."""
    from paper_2512_23027_gb300.binding import SG_MIXED
    prob = w.config("ricker128")
    steps = 2
    s = lib(prob, precision=SG_MIXED)
    assert s.sizes["fp32_precond"] == 1
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    Ur, _, _, its_ref = oracle_run(prob, steps, prob.tol)
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"ricker128: mixed vs oracle rel err {err:.3e}, worst mode {modes:.3e}, iters {its} vs {its_ref}")
    assert err <= BAR_MIXED * prob.tol, err
    assert modes <= BAR_MIXED_MODE * prob.tol, modes
    assert all(r <= prob.tol for r in rr)
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_ref))


def _run_env(lib, prob, precision, steps, env):
    """Set-up and steps with the environment switches set: the step graph is captured at the first
    step, and the launch shapes are read again at that point."""
    import os
    for k, v in env.items():
        os.environ[k] = v
    try:
        s = lib(prob, precision=precision)
        s.step(steps)
        u, (its, rr) = s.field(), s.iters()
        s.close()
    finally:
        for k in env:
            del os.environ[k]
    return u, its, rr


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nods", ["1", "2"])
def test_wide_subdomain_kernel_variants(lib, precision, nods):
    """The kernel variants for subdomains too wide for the shared-memory tiles (runtime-table apply
    that forms the edge differences on the fly, with the triple-product table staged (1) or read
    from global memory (2); line sweep reading the symmetric factor from global memory,
    column-wise) forced on a small problem give the fields of the default kernels: bitwise up to
    the summation order of the factor rows, i.e. within 1e-12 in FP64 and within the solver
    tolerance in mixed precision."""
    prob = w.config("small")
    ua, ia, _ = _run_env(lib, prob, precision, 3, {})
    ub, ib, rb = _run_env(lib, prob, precision, 3, {"SG_FORCE_NODS": nods, "SG_FORCE_GLINE": "1",
                                                    "SG_NO_MMA": "1", "SG_NO_GFIX": "1"})
    err = rel(ub, ua)
    print(f"precision {precision}: forced wide-subdomain variants vs default rel diff {err:.3e}")
    assert err <= (1e-12 if precision == 0 else 1e2 * prob.tol), err
    assert all(r <= prob.tol for r in rb)
    assert all(abs(x - y) <= 1 for x, y in zip(ia, ib))


@pytest.mark.slow
@pytest.mark.parametrize("which", ["240^2 P=10", "256^2 P=35"])
def test_widest_batch_subdomains_converge(lib, which):
    """Batch instances whose subdomains exceed the shared-memory tiles (240^2 grid, 2 x 2
    subdomains of 121 x 121 nodes, P = 10; 256^2 grid, 2 x 2 subdomains of 129 x 129 nodes, P = 35,
    where the FP64 apply reads the triple-product table from global memory) run with the
    wide-subdomain variants: mixed precision converges every step and agrees with the FP64 solver
    on the same GPU to a small multiple of the tolerance."""
    from paper_2512_23027_gb300.binding import SG_FP64, SG_MIXED
    if which == "240^2 P=10":
        prob = [p for p in w.batch_problems(8) if p.N // p.s + 1 > 81][0]
    else:
        prob = [p for p in w.batch_problems(256) if p.N == 256 and p.s == 2 and p.P == 35][0]
    um, im, rm = _run_env(lib, prob, SG_MIXED, 2, {})
    ud, idd, rd = _run_env(lib, prob, SG_FP64, 2, {})
    err = rel(um, ud)
    print(f"{prob.name} ({prob.N}^2, {prob.s}x{prob.s}, P={prob.P}): mixed vs FP64 rel diff {err:.3e}, "
          f"iters {im} vs {idd}")
    assert all(r <= prob.tol for r in rm + rd)
    assert err <= 1e2 * prob.tol, err


@pytest.mark.parametrize("precision", [0, 1, 3], ids=["fp64", "mixed", "bf16"])
def test_wide_line_kernel_matches_block_kernel(lib, precision):
    """Subdomains of 41 x 41 nodes: the register-tiled line sweep (k_line_w, FP64 and FP32), its form
    with the per-line products on the tensor cores (k_line_tc, SG_BF16) and the block kernel with the
    factor staged line by line (SG_LINE_OLD) give the same fields: up to the summation order of the
    factor rows in FP64 (PCG tolerance 1e-13), within the solver tolerance with FP32 solves; the FP64
    fields also match the oracle."""
    prob = w.config("small").replace(name="w41", N=80, s=2, dt=w.cfl_dt(80), tol=1e-13 if precision == 0 else 1e-8)
    ua, ia, ra = _run_env(lib, prob, precision, 3, {})
    ub, ib, rb = _run_env(lib, prob, 1 if precision == 3 else precision, 3, {"SG_LINE_OLD": "1"})
    err = rel(ua, ub)
    print(f"L = 41, {['fp64', 'mixed', '', 'bf16'][precision]}: wide vs block line kernel rel diff {err:.3e}, "
          f"iters {ia} vs {ib}")
    assert err <= (1e-12 if precision == 0 else 1e2 * prob.tol), err
    assert all(r <= prob.tol for r in ra + rb)
    assert all(abs(x - y) <= 1 for x, y in zip(ia, ib))
    if precision == 0:
        Ur, _, _, its_ref = oracle_run(prob, 3, 1e-13)
        assert rel(ua, Ur) <= BAR_U and rel_modes(ua, Ur).max() <= BAR_U_MODE



def _caller_kl(prob):
    """Caller KL: the analytic modes times 1 + 0.3 sin(7x + 3y) at the element centroids (neither
    separable nor symmetric), lambdas 0.37 and 0.11; returns (modes, lambdas, element PCE coefficients
    the oracle builds from them)."""
    from oracle import fem, field, kl
    _, cen = fem.elements(prob.N)
    bump = 1.0 + 0.3 * np.sin(7 * cen[:, 0] + 3 * cen[:, 1])
    lam = np.array([0.37, 0.11])
    phi = np.array([kl.phi1d(cen[:, 0], wx, px) * kl.phi1d(cen[:, 1], wy, py) * bump
                    for _, (ix, wx, px), (iy, wy, py) in kl.kl_modes(prob.M, prob.bx, prob.by)])
    coef = field.lognormal_pce(prob.sigma * np.sqrt(lam)[:, None] * phi, prob.g0, prob.p_in)
    return phi, lam, coef


def test_caller_kl_modes_match_oracle(lib):
    """sg_kl.modes / lambdas: the same caller KL drives the library and the oracle (which builds its
    element coefficients from the same centroid values); FP64 at PCG tolerance 1e-13."""
    prob = w.config("small")
    phi, lam, coef = _caller_kl(prob)
    steps = 3
    s = lib(prob, tol=1e-13, kl_modes=phi, kl_lambdas=lam)
    s.step(steps)
    U = s.field()
    s.close()
    sgp = osg.SGProblem(prob, coef=coef)
    d = odd.DDSolver(prob, coef=coef)
    Ur, _, _, _ = odd.run_dd(sgp, d, steps, tol=1e-13)
    Ur = Ur.reshape(U.shape)
    d0 = osg.SGProblem(prob)
    U0, _, _, _ = odd.run_dd(d0, odd.DDSolver(prob), steps, tol=1e-13)
    print(f"caller KL: rel err {rel(U, Ur):.2e}, worst mode {rel_modes(U, Ur).max():.2e}; differs from the "
          f"analytic-KL field by {rel(U, U0.reshape(U.shape)):.2e}")
    assert rel(U, Ur) <= BAR_U and rel_modes(U, Ur).max() <= BAR_U_MODE
    assert rel(U, U0.reshape(U.shape)) > 1e-4   # the caller's modes were used


@pytest.mark.parametrize("precision", [2, 3], ids=["fp32", "bf16"])
def test_fp32_and_bf16_modes(lib, precision):
    """SG_FP32 (FP32 line sweeps) and SG_BF16 (BF16 tensor-core preconditioner) inside the FP64 outer
    PCG, against the oracle at the workload tolerance."""
    prob = w.config("small")
    steps = 4
    s = lib(prob, precision=precision)
    assert s.sizes["fp32_precond"] == (1 if precision == 3 else 0)
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    Ur, _, _, its_ref = oracle_run(prob, steps, prob.tol)
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"precision {precision}: rel err {err:.2e} ({err / prob.tol:.2f} tol), worst mode {modes:.2e}, "
          f"iters {its} vs {its_ref}")
    assert err <= BAR_MIXED * prob.tol and modes <= BAR_MIXED_MODE * prob.tol
    assert all(r <= prob.tol for r in rr)
    assert all(a <= b + 2 for a, b in zip(its, its_ref))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("pc", [1, 2], ids=["nn1", "lumped"])
def test_one_level_preconditioners_match_oracle(lib, pc, precision):
    """The comparison preconditioners of Sec. 6.1 (one-level Neumann-Neumann: local Neumann solves
    with the whole interface free, no coarse space; lumped: K~_GG on the interface) against the
    oracle's PCG with the same preconditioner: FP64 at PCG tolerance 1e-13, mixed at the workload
    tolerance; outer iteration counts within one of the oracle's."""
    name = {1: "nn1", 2: "lumped"}[pc]
    prob = w.config("small")
    tol = 1e-13 if precision == 0 else prob.tol
    steps = 3
    s = lib(prob, precision=precision, tol=tol, precond=pc)
    s.step(steps)
    U = s.field()
    its, rr = s.iters()
    s.close()
    d = odd.DDSolver(prob, precond=name)
    Ur, _, _, it = odd.run_dd(osg.SGProblem(prob), d, steps, tol=tol)
    Ur = Ur.reshape(U.shape)
    its_ref = [i for i, _ in it]
    err, modes = rel(U, Ur), rel_modes(U, Ur).max()
    print(f"{name} {'fp64' if precision == 0 else 'mixed'}: rel err {err:.2e}, worst mode {modes:.2e}, "
          f"iters {its} vs {its_ref}")
    if precision == 0:
        assert err <= BAR_U and modes <= BAR_U_MODE
    else:
        assert err <= BAR_MIXED * tol and modes <= BAR_MIXED_MODE * tol
    assert all(r <= tol for r in rr)
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_ref))
