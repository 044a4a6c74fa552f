"""Log-normal wave-speed field c_s = exp(g) expanded in Hermite chaos (Sec. 4,
Eqs. c0pce, LNL0).

Reading of Eq. c0pce (garbled in the source): the coefficient of Psi_alpha is
E[exp(g) Psi_alpha(xi)] = c_0(x) prod_n g_n(x)^alpha_n / sqrt(alpha_n!),
with c_0(x) = exp(g0 + 1/2 sum_n g_n(x)^2) the mean (Eq. LNL0), because
E[exp(g xi) He_k(xi)] = g^k exp(g^2/2) for xi ~ N(0, 1).
"""
from __future__ import annotations

import math

import numpy as np

from .pce import multi_indices


def lognormal_pce(gn: np.ndarray, g0: float, p_in: int) -> np.ndarray:
    """gn: (M, npts) KL fields at the points.  Returns c[alpha, pt] for |alpha| <= p_in."""
    M = gn.shape[0]
    c0 = np.exp(g0 + 0.5 * np.sum(gn * gn, axis=0))
    A = multi_indices(M, p_in)
    out = np.zeros((len(A), gn.shape[1]))
    for i, a in enumerate(A):
        term = c0.copy()
        for n in range(M):
            if a[n]:
                term = term * gn[n] ** a[n] / math.sqrt(math.factorial(a[n]))
        out[i] = term
    return out
