"""Run-to-run reproducibility of the mixed-precision step: the step performs no atomics on floating
point values and reduces every partial sum in a fixed order, so two solvers given the same problem
must hold bitwise identical states after every step.  A difference means a kernel read data before
it was written (a race) or read uninitialised memory.

The workload is the 1024^2 problem's subdomain shape and PCE (65 x 65 nodes, M = 5, p = 2) on a
512^2 grid with 8 x 8 subdomains: 64 subdomain problems, so the register-tiled line sweep splits the
21 modes of each problem over two blocks (the register-tiled sweep, or its tensor-core form)."""
import pytest

import sg_workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    return Solver


def test_two_solvers_stay_bitwise_identical(lib):
    import torch
    from paper_2512_23027_gb300.binding import SG_MIXED, plan_query
    prob = w.config("ricker1024q")
    plan = plan_query(prob, SG_MIXED)
    assert plan["line_kind"][1] in (3, 4) and plan["line_groups"][1] == 2, plan
    a = lib(prob, precision=SG_MIXED)
    b = lib(prob, precision=SG_MIXED)
    n = 3 * a.n_free * a.P + 1
    sa = torch.zeros(n, dtype=torch.float64, device="cuda")
    sb = torch.zeros(n, dtype=torch.float64, device="cuda")
    first = None
    for k in range(1, 61):
        a.step(1)
        b.step(1)
        a.get_state(sa)
        b.get_state(sb)
        torch.cuda.synchronize()
        if not torch.equal(sa, sb):
            first = k
            break
    ia, ib = a.iters()[0], b.iters()[0]
    a.close()
    b.close()
    assert first is None, f"states differ after step {first}"
    assert ia == ib
