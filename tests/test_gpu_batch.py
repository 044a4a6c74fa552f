"""Batched solve (sg_solve_batch): several independent problems of different sizes, precisions and
PCE orders advance together in one graph launch.  Each must give exactly the result of stepping it
alone (same kernels, same order within each problem), and the batched workload generator must be
reproducible."""
import numpy as np
import pytest

import sg_workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Solver():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver as S
    return S


@pytest.mark.parametrize("warm", ["prev", "learned"])
def test_batch_equals_individual(Solver, warm):
    """Batched and individual steps agree bitwise, with the previous-step guess and with the learned
    warm start (its statistics, least-squares fit and network training run inside each problem's
    branch of the batch graph)."""
    from paper_2512_23027_gb300 import solve_batch
    from paper_2512_23027_gb300.binding import SG_FP64, SG_MIXED, SG_WARM_LEARNED, SG_WARM_PREV
    wm = SG_WARM_LEARNED if warm == "learned" else SG_WARM_PREV
    probs = [(w.config("small"), SG_FP64), (w.config("tiny"), SG_FP64), (w.config("pulse32"), SG_MIXED),
             (w.config("small").replace(p=3, p_in=3, sigma=0.45), SG_MIXED)]
    steps = 6 if warm == "learned" else 3   # the error history fills after four steps
    batch = [Solver(p, precision=pr, warm=wm) for p, pr in probs]
    stats = solve_batch(batch, steps)
    for (p, pr), s, st in zip(probs, batch, stats):
        ref = Solver(p, precision=pr, warm=wm)
        ref.step(steps)
        assert np.array_equal(s.field(), ref.field()), p.name
        its_b, _ = s.iters()
        its_r, _ = ref.iters()
        assert its_b == its_r
        assert st["step_index"] == steps and st["iters_total"] == sum(its_r)
        ref.close()
    # a second batched call continues from the current state
    solve_batch(batch, 2)
    for (p, pr), s in zip(probs, batch):
        ref = Solver(p, precision=pr, warm=wm)
        ref.step(steps + 2)
        assert np.array_equal(s.field(), ref.field()), p.name
        ref.close()
        s.close()


def test_batch_workload_draw_is_reproducible():
    a = w.batch_problems(256)
    b = w.batch_problems(256)
    assert a == b
    assert all(p.N % p.s == 0 and 64 <= p.N <= 256 and p.s in (2, 4, 8) for p in a)
    assert {p.M for p in a} == {2, 3, 4} and {p.p for p in a} == {2, 3}


def test_autotuned_tiles_match_heuristic_tiles(Solver):
    """Tile shapes chosen by the set-up autotuner change only summation order."""
    prob = w.config("small")
    a = Solver(prob, tol=1e-13)
    a.step(3)
    b = Solver(prob, tol=1e-13, autotune=True)
    b.step(3)
    ua, ub = a.field(), b.field()
    assert np.linalg.norm(ua - ub) <= 1e-10 * np.linalg.norm(ua)
    a.close()
    b.close()
