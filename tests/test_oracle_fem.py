"""Pins for the P1 discretisation and Newmark stepping: element closed forms, mass and
stiffness invariants, the analytic standing wave of the deterministic verification
appendix (O(h^2 + dt^2) convergence of e(t)), and exact energy conservation of the
average-acceleration scheme."""
import json
import math
import os

import numpy as np
import scipy.sparse.linalg as spla

import sg_workloads as w
from oracle import fem, pce, sg

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_newmark_constants_match_paper():
    assert sg.GAMMA == GOLD["newmark_gamma"]["value"]
    assert sg.ZETA == GOLD["newmark_zeta"]["value"]


def test_element_closed_forms():
    h = 0.25
    K, M = fem.element_matrices(np.array([[0.0, 0.0], [h, 0.0], [h, h]]))
    # right angle at the 2nd vertex: legs of unit stiffness 1/2, diagonal edge 0
    assert np.allclose(K, [[0.5, -0.5, 0.0], [-0.5, 1.0, -0.5], [0.0, -0.5, 0.5]])
    assert np.allclose(M, h * h / 24 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]))


def test_mass_and_stiffness_invariants():
    N = 6
    coef = np.ones((1, 2 * N * N))
    M, Ks = fem.assemble(N, coef)
    assert abs(M.sum() - 1.0) < 1e-14                      # total area
    X, Y = fem.node_xy(N)
    assert np.abs(Ks[0] @ np.ones(X.size)).max() < 1e-13    # constants in the kernel
    lin = 2.0 * X - 3.0 * Y + 1.0                           # patch test on interior rows
    r = Ks[0] @ lin
    interior = [fem.node_id(i, j, N) for j in range(1, N) for i in range(1, N)]
    assert np.abs(r[interior]).max() < 1e-12


def test_point_load_reproduces_linears():
    N = 10
    X, Y = fem.node_xy(N)
    for (x, y) in [(0.3, 0.5), (0.37, 0.61), (0.5, 0.5), (0.91, 0.05)]:
        v = fem.p1_values(N, x, y)
        assert abs(sum(v.values()) - 1.0) < 1e-14
        assert abs(sum(val * X[k] for k, val in v.items()) - x) < 1e-14
        assert abs(sum(val * Y[k] for k, val in v.items()) - y) < 1e-14


def standing_wave_error(N, t_end=0.25):
    """Relative error e(t) (Eq. Norm) of the deterministic standing wave, CFL 0.25."""
    m, n, c = GOLD["standing_wave"]["m"], GOLD["standing_wave"]["n"], GOLD["standing_wave"]["c"]
    prob = w.Problem("sw", N=N, s=1, M=1, p=0, p_in=0, sigma=0.0, bx=1, by=1, g0=0.0,
                     dt=0.25 / N, steps=0, tol=0, source=w.Source(), alpha0=0.0, alpha1=0.0)
    coef = fem.element_coefficients(prob)
    Mf, Kf = fem.assemble(N, coef)
    free = fem.free_nodes(N)
    G = pce.triple_products(1, 0, 0)
    ops = sg.SGOperators(Mf[free][:, free], [Kf[0][free][:, free]], G, 0.0, 0.0, prob.dt)
    X, Y = fem.node_xy(N)
    X, Y = X[free], Y[free]
    U = np.sin(m * math.pi * X) * np.sin(n * math.pi * Y)
    V = np.zeros_like(U)
    A = ops.initial_acceleration(np.zeros_like(U), U, V)
    lu = spla.splu(ops.Kt.tocsc())
    steps = int(round(t_end / prob.dt))
    for k in range(steps):
        Ft, um = ops.effective_load(np.zeros_like(U), U, V, A)
        Un = lu.solve(Ft)
        V, A = ops.update(Un, U, V, A, um)
        U = Un
    t = steps * prob.dt
    exact = np.sin(m * math.pi * X) * np.sin(n * math.pi * Y) * math.cos(c * math.pi * math.sqrt(m * m + n * n) * t)
    return np.linalg.norm(exact - U) / np.linalg.norm(exact)


def test_standing_wave_second_order():
    e = [standing_wave_error(N) for N in (8, 16, 32)]
    assert e[2] < 0.03
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.0 < r1 < 5.0 and 3.5 < r2 < 4.5, e


def test_energy_conserved_undamped_sg():
    prob = w.config("tiny").replace(alpha0=0.0, alpha1=0.0, sigma=0.4)
    sgp = sg.SGProblem(prob)
    ops = sgp.ops
    U, V, A = sgp.initial_state()
    lu = spla.splu(ops.Kt.tocsc())
    E0 = 0.5 * V @ (ops.Mb @ V) + 0.5 * U @ (ops.Kb @ U)
    for n in range(40):
        Ft, um = ops.effective_load(np.zeros_like(U), U, V, A)
        Un = lu.solve(Ft)
        V, A = ops.update(Un, U, V, A, um)
        U = Un
        E = 0.5 * V @ (ops.Mb @ V) + 0.5 * U @ (ops.Kb @ U)
        assert abs(E - E0) < 1e-12 * E0


def test_ricker_closed_form_properties():
    """The Ricker wavelet r(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - 1/f: value 1
    at tau = 0, zeros at tau = +-1 / (pi f sqrt 2), zero integral over the line, and equal to
    -1 / (2 pi^2 f^2) times the second derivative of the Gaussian exp(-pi^2 f^2 tau^2)
    (central differences)."""
    for f in (5.0, 10.0, 25.0):
        t0 = 1.0 / f
        assert abs(fem.ricker(t0, f) - 1.0) < 1e-15
        tz = 1.0 / (math.pi * f * math.sqrt(2.0))
        assert abs(fem.ricker(t0 + tz, f)) < 1e-14 and abs(fem.ricker(t0 - tz, f)) < 1e-14
        assert fem.ricker(t0 + 2 * tz, f) < 0 < fem.ricker(t0 + 0.5 * tz, f)
        ts = np.linspace(t0 - 10.0 / f, t0 + 10.0 / f, 20001)
        vals = np.array([fem.ricker(t, f) for t in ts])
        dtq = ts[1] - ts[0]
        assert abs(np.sum(vals) * dtq) < 1e-12 / f
        gauss = lambda t: math.exp(-(math.pi * f * (t - t0)) ** 2)
        hq = 1e-4 / f
        for t in (t0 - 0.3 / f, t0 + 0.05 / f, t0 + 0.7 / f):
            d2 = (gauss(t + hq) - 2 * gauss(t) + gauss(t - hq)) / hq ** 2
            assert abs(-d2 / (2 * math.pi ** 2 * f ** 2) - fem.ricker(t, f)) < 1e-6


def test_point_source_load_taken_at_the_new_time_level():
    """Newmark solves for u_{n+1} with the load at t_{n+1} (Sec. 2, Eq. fparts).  Against an
    independent high-order integration (scipy DOP853) of the semi-discrete system
    M u'' + C u' + K u = f(t) with the Ricker point source, the error of the time-stepped solution
    falls by 4 per halving of dt; taking the load at t_n instead would give a ratio of 2."""
    from scipy.integrate import solve_ivp
    prob = w.config("small").replace(N=4, s=1, M=1, p=0, p_in=0, sigma=0.0)
    T = 0.25
    sgp = sg.SGProblem(prob)
    M, C, K = (x.toarray() for x in (sgp.ops.Mb, sgp.ops.Cb, sgp.ops.Kb))
    Minv = np.linalg.inv(M)
    n = M.shape[0]

    def rhs(t, y):
        u, v = y[:n], y[n:]
        return np.concatenate([v, Minv @ (sgp.load(t) - C @ v - K @ u)])

    ue = solve_ivp(rhs, (0.0, T), np.zeros(2 * n), method="DOP853", rtol=1e-12, atol=1e-15).y[:n, -1]
    errs = []
    for ns in (50, 100, 200):
        U, _, _ = sg.run_direct(sg.SGProblem(prob.replace(dt=T / ns)), ns)
        errs.append(np.linalg.norm(U - ue) / np.linalg.norm(ue))
    assert errs[-1] < 2e-4
    for a, b in zip(errs, errs[1:]):
        assert 3.7 < a / b < 4.3, errs
