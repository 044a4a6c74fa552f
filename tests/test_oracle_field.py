"""Pins for the log-normal PCE (Eqs. c0pce, LNL0 read as the Hermite projection of
exp(g)): pointwise convergence to exp(g0 + sum g_n xi_n) and the closed-form log-normal
mean and variance."""
import math

import numpy as np
from numpy.polynomial import hermite_e as He

from oracle import field, pce


def eval_pce(coef, M, p, xi):
    A = pce.multi_indices(M, p)
    out = 0.0
    for a, c in zip(A, coef):
        term = c
        for n in range(M):
            cc = np.zeros(a[n] + 1)
            cc[a[n]] = 1.0
            term *= He.hermeval(xi[n], cc) / math.sqrt(math.factorial(a[n]))
        out += term
    return out


def test_pointwise_convergence():
    gn = np.array([[0.3], [-0.2]])
    xi = np.array([0.7, -1.1])
    exact = math.exp(0.1 + 0.3 * 0.7 - 0.2 * -1.1)
    errs = []
    for p in (2, 4, 6, 8, 10):
        c = field.lognormal_pce(gn, 0.1, p)[:, 0]
        errs.append(abs(eval_pce(c, 2, p, xi) - exact))
    assert errs[-1] < 1e-9 * exact
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_mean_and_variance_closed_form():
    gn = np.array([[0.4], [0.25], [-0.1]])
    s2 = float(np.sum(gn ** 2))
    c = field.lognormal_pce(gn, 0.0, 12)[:, 0]
    assert abs(c[0] - math.exp(0.5 * s2)) < 1e-15
    var = np.sum(c[1:] ** 2)
    exact = math.exp(s2) * (math.exp(s2) - 1.0)
    assert abs(var - exact) < 1e-12 * exact
