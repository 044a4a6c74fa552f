"""Host-only launch plans (sg_plan_query: the problem is built on the host, no GPU is used) of the
named workloads and of every instance of the 256-problem batch, in both precisions.  Every
per-step kernel must launch within the device limits: blocks of whole warps and at most 1024
threads, dynamic shared memory within the limit the library opts each kernel into, tiles that cover
the subdomain, and a tensor-core tiling whose 128-row tiles and 64-node chunks cover the L^2 nodes
of a subdomain (the last chunk may hold none)."""
import pytest

import sg_workloads as w

SMEM_OPTIN = 232448 - 1024   # opt-in dynamic shared memory per block used by the widest variants
SMEM_DEFAULT = 200 * 1024    # limit of the other variants
SMEM_BLOCK = 232448          # per-block total on the device (dynamic + static)
SG_FP64, SG_MIXED = 0, 1


@pytest.fixture(scope="module")
def plan_query():
    from paper_2512_23027_gb300 import build as b
    b.build()
    from paper_2512_23027_gb300.binding import plan_query
    return plan_query


def problems():
    named = [w.config(n) for n in ("tiny", "small", "pulse32", "ricker128", "ricker512", "ricker1024")]
    return named + w.batch_problems(256)


def check_plan(p, prob, precision):
    L = prob.N // prob.s + 1
    assert (p["L"], p["P"], p["nsub"]) == (L, prob.P, prob.s * prob.s)
    assert p["fits"] == 1
    # kernels the precision launches: the FP64 apply always (residual corrections in mixed mode),
    # the FP32 apply and line sweep in mixed mode, the FP64 line sweep in FP64 mode
    applies = (0, 1) if precision == SG_MIXED else (0,)
    lines = (1,) if precision == SG_MIXED else (0,)
    for i in applies:  # 0: FP64 kernels, 1: FP32 kernels
        tl, nt = p["apply_lines"][i], p["apply_tiles"][i]
        assert 1 <= tl <= L and nt == -(-L // tl)
        cap = SMEM_OPTIN if p["apply_variant"][i] == 2 else SMEM_DEFAULT
        assert 0 < p["apply_smem"][i] <= cap
        if p["apply_variant"][i] == 3:  # compiled table: only where a one-line tile fits
            assert p["P"] == prob.P and p["P_in"] == prob.P_in
    for i in lines:
        threads = p["line_block"][i][0] * p["line_block"][i][1] * p["line_block"][i][2]
        assert 32 <= threads <= 1024 and threads % 32 == 0
        g, ng = p["line_modes"][i], p["line_groups"][i]
        assert g * ng >= prob.P and (ng - 1) * g < prob.P
        cap = SMEM_OPTIN if p["line_kind"][i] == 1 else SMEM_DEFAULT
        assert 0 < p["line_smem"][i] <= cap
        if p["line_kind"][i] == 3:  # register-tiled sweep of wide subdomains: <= 256 threads, 2 x 4 tiles
            assert L >= 41 and threads <= 256
            gs = -(-g // 4) * 4
            lsp = -(-L // 4) * 4
            assert threads >= (lsp // 2) * (gs // 4)
    expect_mma = precision == SG_MIXED and L <= 40 and prob.P <= 32
    assert p["mma"] == int(expect_mma)
    if expect_mma:
        kp = p["mma_kp"]
        assert kp % 128 == 0 and L * L <= kp < L * L + 128
        assert p["mma_nc"] * 64 == kp and p["mma_mt"] * 128 == kp
        assert p["mma_nb"] in (16, 32) and prob.P <= p["mma_nb"] and (p["mma_nb"] == 16) == (prob.P <= 16)
        assert 0 < p["mma_smem"] and p["mma_smem"] + 1024 <= SMEM_BLOCK


@pytest.mark.parametrize("precision", [SG_FP64, SG_MIXED])
def test_every_workload_and_batch_instance_has_a_valid_plan(plan_query, precision):
    n_mma = n_gtab = 0
    for prob in problems():
        p = plan_query(prob, precision)
        check_plan(p, prob, precision)
        n_mma += p["mma"]
        n_gtab += p["apply_variant"][0] == 2
    if precision == SG_MIXED:
        assert n_mma > 100  # the tensor-core preconditioner covers most batch instances
    assert n_gtab >= 1      # the 256^2 / 2 x 2 / P = 35 instance needs the global-table FP64 apply


def test_plan_rejects_invalid_sizes(plan_query):
    from paper_2512_23027_gb300.binding import SGError
    prob = w.config("small")
    with pytest.raises(SGError) as e:
        plan_query(prob.replace(N=25), SG_FP64)  # 25 cells do not split into 3 equal subdomains
    assert e.value.code == -1
    with pytest.raises(SGError) as e:
        plan_query(prob, 7)  # unknown precision
    assert e.value.code == -1


# subdomain widths around the thresholds where kernel variants switch (tensor-core preconditioner
# and warp-team line kernel up to 40 nodes, the wide-subdomain variants near 81, 121 and 129 nodes)
SWEEP_H = (3, 15, 19, 38, 39, 40, 41, 63, 64, 80, 81, 120, 128)
SWEEP_MP = ((1, 3), (2, 4), (3, 3), (4, 3), (6, 2))   # P = 4, 15, 20, 35, 28


def test_plans_at_size_thresholds(plan_query):
    from paper_2512_23027_gb300.binding import SGError
    base = w.config("ricker128")
    n_fit = 0
    for H in SWEEP_H:
        for s in ((2, 4) if H <= 64 else (2,)):
            for M, p in SWEEP_MP:
                for precision in (SG_FP64, SG_MIXED):
                    prob = base.replace(N=s * H, s=s, M=M, p=p, p_in=p, dt=w.cfl_dt(s * H))
                    try:
                        plan = plan_query(prob, precision)
                    except SGError as e:
                        assert e.code == -7  # SG_ENOTSUP: outside the build's sizes, never a bad plan
                        continue
                    if plan["fits"]:
                        check_plan(plan, prob, precision)
                        n_fit += 1
                    else:
                        assert precision == SG_FP64 or H > 128
    assert n_fit >= 200
