"""Pins for the Hermite chaos part of the oracle: triple products against Gauss-Hermite
quadrature (an independent evaluation of the integral), closed-form special values and
the PCE sizes printed in the paper."""
import json
import math
import os

import numpy as np
from numpy.polynomial import hermite_e as He

from oracle import pce

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def psi(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return He.hermeval(x, c) / math.sqrt(math.factorial(n))


def test_triple_1d_matches_gauss_hermite():
    x, w = He.hermegauss(20)
    w = w / math.sqrt(2 * math.pi)  # probability measure of N(0,1)
    for a in range(7):
        for b in range(7):
            for c in range(7):
                quad = np.sum(w * psi(a, x) * psi(b, x) * psi(c, x))
                assert abs(pce.hermite_triple_1d(a, b, c) - quad) < 1e-11, (a, b, c)


def test_special_values():
    assert abs(pce.hermite_triple_1d(1, 1, 2) - math.sqrt(2)) < 1e-15
    assert abs(pce.hermite_triple_1d(2, 2, 2) - 2 * math.sqrt(2)) < 1e-14
    assert pce.hermite_triple_1d(1, 1, 1) == 0.0
    assert pce.hermite_triple_1d(0, 3, 1) == 0.0


def test_multi_index_counts_match_paper():
    for M, p, P in GOLD["pce_terms"]["value"]:
        assert len(pce.multi_indices(M, p)) == P
    assert pce.multi_indices(2, 2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]


def test_multivariate_triple_products_by_tensor_quadrature():
    M, p_in, p = 2, 2, 3
    G = pce.triple_products(M, p_in, p)
    x, w = He.hermegauss(12)
    w = w / math.sqrt(2 * math.pi)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    A_in, A_out = pce.multi_indices(M, p_in), pce.multi_indices(M, p)
    ev = lambda a: psi(a[0], X1) * psi(a[1], X2)
    for i, ai in enumerate(A_in):
        for j, aj in enumerate(A_out):
            for k, ak in enumerate(A_out):
                assert abs(G[i, j, k] - np.sum(W * ev(ai) * ev(aj) * ev(ak))) < 1e-11


def test_structure():
    G = pce.triple_products(3, 3, 3)
    assert np.allclose(G, np.transpose(G, (0, 2, 1)))
    assert np.array_equal(G[0], np.eye(G.shape[1]))
    # a first-order i couples only modes whose degrees differ by one
    A = pce.multi_indices(3, 3)
    deg = np.array([sum(a) for a in A])
    for j in range(len(A)):
        for k in range(len(A)):
            if G[1, j, k] != 0:
                assert abs(deg[j] - deg[k]) == 1
