"""Karhunen-Loeve expansion of the Gaussian field g (Sec. 4, Eqs. CovarKer2D, KLE).

Covariance sigma^2 exp(-|x1-x2|/bx - |y1-y2|/by) on the unit square.  The kernel is
separable, so 2-D eigenpairs are products of 1-D ones.  The 1-D kernel exp(-c|x-y|) on
[-a, a] (here a = 1/2, c = 1/b) has the classical analytic eigenpairs:
  even: c - w tan(w a) = 0,   phi = cos(w u) / sqrt(a + sin(2 w a) / (2 w))
  odd : w + c tan(w a) = 0,   phi = sin(w u) / sqrt(a - sin(2 w a) / (2 w))
  lambda = 2 c / (w^2 + c^2),  u = x - 1/2.
The paper states only the expansion; ordering of tied 2-D eigenvalues is a reading:
descending lambda, ties broken by the lower y-index first, then the lower x-index.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.optimize import brentq


def eig1d(b: float, n: int) -> List[Tuple[float, float, int]]:
    """First n 1-D eigenpairs as (lambda, omega, parity) with parity 0 = even (cos),
    1 = odd (sin), in ascending omega (descending lambda)."""
    c = 1.0 / b
    a = 0.5
    out = []
    k = 0
    while len(out) < n:
        lo, hi = 2 * k * math.pi, 2 * k * math.pi + math.pi
        f_even = lambda w: c - w * math.tan(w * a)
        w = brentq(f_even, lo + 1e-10, hi - 1e-10, xtol=1e-15, rtol=1e-15, maxiter=500)
        out.append((2 * c / (w * w + c * c), w, 0))
        if len(out) == n:
            break
        lo, hi = 2 * k * math.pi + math.pi, 2 * k * math.pi + 2 * math.pi
        f_odd = lambda w: w + c * math.tan(w * a)
        w = brentq(f_odd, lo + 1e-10, hi - 1e-10, xtol=1e-15, rtol=1e-15, maxiter=500)
        out.append((2 * c / (w * w + c * c), w, 1))
        k += 1
    return out


def phi1d(x, w: float, parity: int):
    u = np.asarray(x, dtype=float) - 0.5
    if parity == 0:
        return np.cos(w * u) / math.sqrt(0.5 + math.sin(w) / (2 * w))
    return np.sin(w * u) / math.sqrt(0.5 - math.sin(w) / (2 * w))


def kl_modes(M: int, bx: float, by: float):
    """Top-M 2-D modes: list of (lambda, (ix, wx, px), (iy, wy, py))."""
    ex = eig1d(bx, M + 1)
    ey = eig1d(by, M + 1)
    cand = []
    for ix, (lx, wx, px) in enumerate(ex):
        for iy, (ly, wy, py) in enumerate(ey):
            cand.append((lx * ly, iy, ix, (ix, wx, px), (iy, wy, py)))
    cand.sort(key=lambda t: (-t[0], t[1], t[2]))
    return [(t[0], t[3], t[4]) for t in cand[:M]]


def kl_fields(M: int, sigma: float, bx: float, by: float, x, y) -> np.ndarray:
    """g_n(x) = sigma sqrt(lambda_n) phi_n(x) for n < M at points (x, y); shape (M, npts)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    out = np.zeros((M, x.size))
    for n, (lam, (ix, wx, px), (iy, wy, py)) in enumerate(kl_modes(M, bx, by)):
        out[n] = sigma * math.sqrt(lam) * phi1d(x, wx, px) * phi1d(y, wy, py)
    return out
