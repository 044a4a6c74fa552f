"""Hermite polynomial chaos: multi-indices and triple products (Sec. 4).

Basis: normalised probabilists' Hermite polynomials psi_n = He_n / sqrt(n!), so that
<Psi_i Psi_j> = delta_ij (Eq. PCEOrtho with the normalisation stated in Sec. 6).
Multivariate Psi_alpha(xi) = prod_d psi_{alpha_d}(xi_d).
"""
from __future__ import annotations

import math
from itertools import product
from typing import List, Tuple

import numpy as np


def multi_indices(M: int, p: int) -> List[Tuple[int, ...]]:
    """All alpha in N^M with |alpha| <= p, graded by total degree; within a degree in
    descending lexicographic order (xi1^2 before xi1 xi2 before xi2^2).  The paper does
    not fix an order; results are invariant under a permutation of the modes."""
    out: List[Tuple[int, ...]] = []
    for d in range(p + 1):
        level = [a for a in product(range(d + 1), repeat=M) if sum(a) == d]
        level.sort(reverse=True)
        out.extend(level)
    return out


def hermite_triple_1d(a: int, b: int, c: int) -> float:
    """<psi_a psi_b psi_c> for normalised probabilists' Hermite polynomials.

    Closed form: <He_a He_b He_c> = a! b! c! / ((s-a)! (s-b)! (s-c)!) when
    s = (a+b+c)/2 is an integer with s >= max(a,b,c), else 0; dividing by
    sqrt(a! b! c!) normalises.
    """
    if (a + b + c) % 2:
        return 0.0
    s = (a + b + c) // 2
    if s < a or s < b or s < c:
        return 0.0
    num = math.sqrt(math.factorial(a) * math.factorial(b) * math.factorial(c))
    den = math.factorial(s - a) * math.factorial(s - b) * math.factorial(s - c)
    return num / den


def triple_products(M: int, p_in: int, p: int) -> np.ndarray:
    """Dense G[i, j, k] = <Psi_i Psi_j Psi_k> (Sec. 4, G_ijk), i over the input basis
    (order p_in), j, k over the output basis (order p)."""
    A_in = multi_indices(M, p_in)
    A_out = multi_indices(M, p)
    G = np.zeros((len(A_in), len(A_out), len(A_out)))
    for i, ai in enumerate(A_in):
        for j, aj in enumerate(A_out):
            for k, ak in enumerate(A_out):
                v = 1.0
                for d in range(M):
                    v *= hermite_triple_1d(ai[d], aj[d], ak[d])
                    if v == 0.0:
                        break
                G[i, j, k] = v
    return G
