"""Monte Carlo reference for the stochastic wave problem (Sec. 6.2 verification of the
SG method against MCS; standard error from the central limit theorem, 1-D bar appendix).

Per sample xi ~ N(0, I_M): a deterministic FE problem with the exact log-normal
coefficient c(x_e, xi) = exp(g0 + sum_n g_n(x_e) xi_n) at element centroids (not its
PCE), the same Newmark-beta scheme, a direct solve per step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem, kl
from .sg import SGOperators


def mc_moments(prob, xis: np.ndarray, steps: int):
    """Mean and variance (over the samples) of the nodal solution on the free nodes
    after `steps` steps; xis is (n_samples, M)."""
    N = prob.N
    _, cen = fem.elements(N)
    gn = kl.kl_fields(prob.M, prob.sigma, prob.bx, prob.by, cen[:, 0], cen[:, 1])
    free = fem.free_nodes(N)
    G1 = np.ones((1, 1, 1))
    s1 = np.zeros(free.size)
    s2 = np.zeros(free.size)
    for xi in xis:
        c = np.exp(prob.g0 + gn.T @ xi)[None, :]
        Mf, Kf = fem.assemble(N, c)
        M = Mf[free][:, free]
        K = Kf[0][free][:, free]
        ops = SGOperators(M, [K], G1, prob.alpha0, prob.alpha1, prob.dt)
        lu = spla.splu(ops.Kt.tocsc())
        U = fem.initial_displacement(N, prob.source)[free]
        V = np.zeros_like(U)
        F0 = fem.point_load(N, prob.source, 0.0)[free]
        A = ops.initial_acceleration(F0, U, V)
        for n in range(steps):
            t = (n + 1) * prob.dt
            Ft, um = ops.effective_load(fem.point_load(N, prob.source, t)[free], U, V, A)
            Un = lu.solve(Ft)
            V, A = ops.update(Un, U, V, A, um)
            U = Un
        s1 += U
        s2 += U * U
    n = xis.shape[0]
    mean = s1 / n
    var = (s2 - n * mean * mean) / (n - 1)
    return mean, var
