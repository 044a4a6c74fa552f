"""sg_setup rejects invalid and unsupported inputs before it touches the GPU (no device needed):
every failure returns its status code (SG_EINVAL -1, SG_ENOTSUP -7) with a message in
sg_last_error(NULL), leaves the output handle NULL, and issues no CUDA call (the checks run before
the first one), so these tests run on a machine without a GPU."""
import ctypes as C

import pytest

import sg_workloads as w

SG_EINVAL, SG_ENOTSUP = -1, -7


@pytest.fixture(scope="module")
def B():
    from paper_2512_23027_gb300 import build as b
    b.build()
    from paper_2512_23027_gb300 import binding
    binding.load_library()
    return binding


def setup_rc(B, prob, precision=0, warm=0, warm_train_steps=0, grid=None, src_kind=None, modes=None, lambdas=None,
             precond=0):
    lib = B.load_library()
    s = prob.source
    g = grid or B.Grid(prob.N, prob.s, prob.s)
    kl = B.KL(prob.M, prob.sigma, prob.bx, prob.by, prob.g0, None if modes is None else modes.ctypes.data,
              None if lambdas is None else lambdas.ctypes.data)
    pce = B.PCE(prob.p, prob.p_in)
    prm = B.Params(prob.dt, prob.tol, prob.alpha0, prob.alpha1, prob.max_iter, precision, warm, 0.0, 0, 0,
                   warm_train_steps, 0.0, precond)
    src = B.Source(s.kind if src_kind is None else src_kind, s.x0, s.y0, s.width, s.freq, s.amp)
    h = C.c_void_p(12345)
    rc = lib.sg_setup(C.byref(g), C.byref(kl), C.byref(pce), C.byref(prm), C.byref(src), None, C.byref(h))
    return rc, h.value, lib.sg_last_error(None).decode()


CASES = [
    ("source kind", dict(src_kind=5), SG_EINVAL, "source"),
    ("precision", dict(precision=7), SG_EINVAL, "precision"),
    ("negative precision", dict(precision=-1), SG_EINVAL, "precision"),
    ("preconditioner", dict(precond=3), SG_EINVAL, "precond"),
    ("warm-start mode", dict(warm=9), SG_EINVAL, "warm"),
    ("warm-start training steps", dict(warm_train_steps=-1), SG_EINVAL, "warm"),
]
PROBS = [
    ("N not divisible by s", dict(N=25), SG_EINVAL, "divisible"),
    ("negative time step", dict(dt=-1e-3), SG_EINVAL, "dt"),
    ("negative sigma", dict(sigma=-0.1), SG_EINVAL, "sigma"),
    ("zero correlation length", dict(bx=0.0), SG_EINVAL, "correlation"),
    ("too many random variables", dict(M=13), SG_EINVAL, "unsupported"),
    ("single subdomain", dict(N=24, s=1), SG_ENOTSUP, "2 x 2"),
    ("subdomains wider than 255 cells", dict(N=512, s=2), SG_ENOTSUP, "255"),
    ("pulse of zero width", dict(source=w.Source(1, 0.5, 0.5, 0.0, 0.0, 1.0)), SG_EINVAL, "width"),
    ("Ricker source outside the square", dict(source=w.Source(2, 1.5, 0.5, 0.0, 10.0, 1.0)), SG_EINVAL, "ricker"),
]


@pytest.mark.parametrize("what,kw,code,msg", CASES, ids=[c[0] for c in CASES])
def test_invalid_parameters(B, what, kw, code, msg):
    rc, h, err = setup_rc(B, w.config("small"), **kw)
    assert rc == code and h is None, (what, rc, err)
    assert msg in err.lower() or msg in err, err


@pytest.mark.parametrize("what,kw,code,msg", PROBS, ids=[c[0] for c in PROBS])
def test_invalid_or_unsupported_problems(B, what, kw, code, msg):
    rc, h, err = setup_rc(B, w.config("small").replace(**kw))
    assert rc == code and h is None, (what, rc, err)
    assert msg.lower() in err.lower(), err


def test_unequal_partition_and_null_arguments(B):
    rc, h, err = setup_rc(B, w.config("small"), grid=B.Grid(24, 3, 2))
    assert rc == SG_EINVAL and h is None and "nsub" in err
    lib = B.load_library()
    out = C.c_void_p(1)
    assert lib.sg_setup(None, None, None, None, None, None, C.byref(out)) == SG_EINVAL
    assert out.value is None


def test_solver_raises_the_status(B):
    with pytest.raises(B.SGError) as e:
        B.Solver(w.config("small").replace(N=25))
    assert e.value.code == SG_EINVAL


def _modes(prob, value=0.5):
    import numpy as np
    return np.full(prob.M * 2 * prob.N * prob.N, value)


def test_caller_kl_arrays_are_checked(B):
    """modes without lambdas, a non-positive lambda and a non-finite mode value are argument errors."""
    import numpy as np
    prob = w.config("small")
    m = _modes(prob)
    rc, h, err = setup_rc(B, prob, modes=m)
    assert rc == SG_EINVAL and h is None and "lambdas" in err
    rc, h, err = setup_rc(B, prob, modes=m, lambdas=np.array([0.3, -0.1]))
    assert rc == SG_EINVAL and h is None and "lambda" in err
    bad = m.copy()
    bad[7] = np.nan
    rc, h, err = setup_rc(B, prob, modes=bad, lambdas=np.array([0.3, 0.1]))
    assert rc == SG_EINVAL and h is None and "finite" in err


def test_bf16_mode_needs_the_tensor_core_preconditioner(B):
    """SG_BF16 requires a BF16 tensor-core mean preconditioner: the dense inverse (subdomains of at most
    40 x 40 nodes, P <= 32) or the line sweeps with per-line tensor-core products (41 .. 65 nodes per
    side).  Wider subdomains get SG_ENOTSUP (before any CUDA call)."""
    prob = w.config("small").replace(N=160, s=2)   # 81 x 81-node subdomains
    rc, h, err = setup_rc(B, prob, precision=3)
    assert rc == SG_ENOTSUP and h is None and "BF16" in err


def test_bf16_line_products_in_the_launch_plan(B):
    """41 x 41- and 65 x 65-node subdomains: SG_BF16 plans the line sweeps with tensor-core products
    (line kind 4, no dense inverse), SG_MIXED and SG_FP32 the register-tiled FP32 sweeps (kind 3)."""
    for N, s in ((80, 2), (128, 2)):
        prob = w.config("small").replace(N=N, s=s)
        plans = {p: B.plan_query(prob, p) for p in (1, 2, 3)}
        assert plans[3]["line_kind"][1] == 4 and plans[3]["mma"] == 0, plans[3]
        assert plans[1]["line_kind"][1] == 3 and plans[2]["line_kind"][1] == 3
        assert plans[3]["line_block"][1][0] % 32 == 0 and plans[3]["line_block"][1][0] >= 128
        assert all(pl["fits"] == 1 for pl in plans.values())


def test_precision_modes_in_the_launch_plan(B):
    """sg_plan_query: SG_MIXED and SG_BF16 take the tensor-core preconditioner on 9 x 9-node
    subdomains, SG_FP32 the line sweeps; every mode launches the FP32 kernels there."""
    prob = w.config("small")
    plans = {p: B.plan_query(prob, p) for p in (1, 2, 3)}
    assert plans[1]["mma"] == 1 and plans[3]["mma"] == 1 and plans[2]["mma"] == 0
    assert all(pl["fits"] == 1 for pl in plans.values())

