"""Pins for the stochastic Galerkin system: the sigma = 0 reduction to the deterministic
solver, a single-dof problem whose exact moments follow from Gauss-Hermite quadrature of
the per-sample Newmark recurrence (brute force in the random variable), and Monte Carlo
agreement within the CLT standard error on a tiny mesh (Sec. 6.2 method)."""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import sg_workloads as w
from oracle import field, mc, pce, sg


def test_sigma_zero_reduces_to_deterministic():
    prob = w.config("tiny").replace(sigma=0.0)
    U, V, A = sg.run_direct(sg.SGProblem(prob), 6)
    P = prob.P
    Um = U.reshape(-1, P)
    assert np.all(Um[:, 1:] == 0.0)
    det = prob.replace(M=1, p=0, p_in=0)
    Ud, _, _ = sg.run_direct(sg.SGProblem(det), 6)
    assert np.abs(Um[:, 0] - Ud).max() < 1e-13 * np.abs(Ud).max()


def single_dof_sg(sigma, p, dt, steps, a0, a1):
    coef = field.lognormal_pce(np.array([[sigma]]), 0.0, p)[:, 0]
    G = pce.triple_products(1, p, p)
    M = sp.csr_matrix([[1.0]])
    Ks = [sp.csr_matrix([[c]]) for c in coef]
    ops = sg.SGOperators(M, Ks, G, a0, a1, dt)
    P = G.shape[1]
    U = np.zeros(P); U[0] = 1.0
    V = np.zeros(P)
    A = ops.initial_acceleration(np.zeros(P), U, V)
    lu = spla.splu(ops.Kt.tocsc())
    for _ in range(steps):
        Ft, um = ops.effective_load(np.zeros(P), U, V, A)
        Un = lu.solve(Ft)
        V, A = ops.update(Un, U, V, A, um)
        U = Un
    return U[0], np.sum(U[1:] ** 2)


def single_dof_exact(sigma, dt, steps, a0, a1):
    x, wq = np.polynomial.hermite_e.hermegauss(80)
    wq = wq / math.sqrt(2 * math.pi)
    g, z = sg.GAMMA, sg.ZETA
    vals = []
    for xi in x:
        k = math.exp(sigma * xi)
        c = a0 + a1 * k
        u, v = 1.0, 0.0
        a = -(c * v + k * u)
        Kt = 1 / (z * dt * dt) + c * g / (z * dt) + k
        for _ in range(steps):
            um = (u + dt * v) / (z * dt * dt) + (1 - 2 * z) * a / (2 * z)
            uc = g * dt * um - v - (1 - g) * a * dt
            un = (um + c * uc) / Kt
            an = un / (z * dt * dt) - um
            v = v + dt * ((1 - g) * a + g * an)
            u, a = un, an
        vals.append(u)
    vals = np.array(vals)
    mean = np.sum(wq * vals)
    return mean, np.sum(wq * (vals - mean) ** 2)


def test_single_dof_converges_to_quadrature():
    sigma, dt, steps, a0, a1 = 0.3, 0.1, 25, 0.05, 0.01
    m_ex, v_ex = single_dof_exact(sigma, dt, steps, a0, a1)
    errs = []
    for p in (2, 4, 6, 8):
        m, v = single_dof_sg(sigma, p, dt, steps, a0, a1)
        errs.append(abs(m - m_ex) + abs(v - v_ex))
    assert errs[-1] < 1e-7
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs


def test_monte_carlo_within_standard_error():
    prob = w.Problem("mc", N=8, s=2, M=2, p=3, p_in=3, sigma=0.3, bx=0.5, by=0.5, g0=0.0,
                     dt=0.02, steps=8, tol=1e-12, source=w.Source(w.SOURCE_PULSE, 0.5, 0.5, 0.2, 0, 1.0))
    U, _, _ = sg.run_direct(sg.SGProblem(prob), prob.steps)
    Um = U.reshape(-1, prob.P)
    sg_mean, sg_var = Um[:, 0], np.sum(Um[:, 1:] ** 2, axis=1)
    n = 2000
    xis = np.array(w.normal_samples(n, prob.M, seed=7))
    mean, var = mc.mc_moments(prob, xis, prob.steps)
    se = np.sqrt(var / n)
    k = np.argmax(np.abs(sg_mean))
    assert np.all(np.abs(sg_mean - mean) <= 4 * se + 1e-12)
    # variance: SE of the sample variance ~ var * sqrt(2 / (n - 1)) for near-Gaussian output
    assert abs(sg_var[k] - var[k]) <= 4 * var[k] * math.sqrt(2.0 / (n - 1)) + 1e-12


def test_matrix_form_operators_equal_the_block_matrices():
    """The matrix-form operators used for full-size checks (oracle.sg.SGMatrixForm) equal the
    Kronecker block matrices of SGOperators (Eq. K_T_Sto, damping of the Rayleigh appendix) on a small
    problem with p_in = 2p, and the direct solve's step leaves a residual at the rounding level."""
    import numpy as np
    import sg_workloads as w
    from oracle import sg
    prob = w.config("tiny").replace(p_in=4, alpha0=0.3, alpha1=0.01)
    sgp = sg.SGProblem(prob)
    ops = sgp.ops
    mf = sg.SGMatrixForm(sgp.M, sgp.Ks, sgp.G, prob.alpha0, prob.alpha1, prob.dt)
    rng = np.random.default_rng(5)
    n, P = sgp.free.size, sgp.P
    X = rng.standard_normal((n, P))
    x = X.ravel()
    for a, b in ((mf.stiffness(X), ops.Kb @ x), (mf.damping(X), ops.Cb @ x), (mf.transient(X), ops.Kt @ x)):
        assert np.abs(a.ravel() - b).max() <= 1e-12 * np.abs(b).max()
    U, V, A = sgp.initial_state()
    F = sgp.load(prob.dt)
    Ft, um = ops.effective_load(F, U, V, A)
    Ft2, um2 = mf.effective_load(F.reshape(n, P), U.reshape(n, P), V.reshape(n, P), A.reshape(n, P))
    assert np.abs(Ft2.ravel() - Ft).max() <= 1e-12 * np.abs(Ft).max() and np.allclose(um2.ravel(), um)
    import scipy.sparse.linalg as spla
    Unew = spla.spsolve(ops.Kt.tocsc(), Ft)
    r = mf.residual(F.reshape(n, P), U.reshape(n, P), V.reshape(n, P), A.reshape(n, P), Unew.reshape(n, P))
    assert r < 1e-13
    # a perturbed solution shows up in the residual
    assert mf.residual(F.reshape(n, P), U.reshape(n, P), V.reshape(n, P), A.reshape(n, P),
                       Unew.reshape(n, P) * (1 + 1e-6)) > 1e-8
