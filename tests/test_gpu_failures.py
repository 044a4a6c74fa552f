"""Failure reporting on the GPU, in the allowed forms (nothing faults, traps or hangs a GPU): a step
that reaches the outer iteration cap returns SG_ENOTCONV with the state advanced, and a non-finite
value in the host-given load of sg_step_host makes the PCG's breakdown check return SG_ENUMERIC."""
import numpy as np
import pytest

import sg_workloads as w

pytestmark = pytest.mark.gpu

SG_ENOTCONV, SG_ENUMERIC = -4, -5


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    return Solver


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_outer_iteration_cap_reports_not_converged(lib, precision):
    prob = w.config("small")
    s = lib(prob, precision=precision, max_iter=1)
    st = s.step(2, allow_notconv=True)
    its, rr = s.iters()
    U = s.field()
    s.close()
    assert st["rc"] == SG_ENOTCONV
    assert st["step_index"] == 2           # the state advanced anyway
    assert its == [1, 1] and all(r > prob.tol for r in rr)
    assert np.all(np.isfinite(U)) and np.abs(U).max() > 0


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_non_finite_host_load_reports_numeric_breakdown(lib, precision):
    from paper_2512_23027_gb300.binding import SGError
    prob = w.config("small").replace(source=w.Source())
    s = lib(prob, precision=precision)
    f = np.zeros((1, s.n_free))
    f[0, s.n_free // 2] = np.nan
    u = np.zeros((1, s.n_free))
    with pytest.raises(SGError) as e:
        s.step_host(1, f, u)
    s.close()
    assert e.value.code == SG_ENUMERIC
