"""P1 finite elements on the structured triangulated unit square (Sec. 2 weak form,
semi-discretisation M u'' + C u' + K u = f).

Grid: N x N cells of side h = 1/N, each split along the diagonal (i,j)->(i+1,j+1) into
T1 = {(i,j), (i+1,j), (i+1,j+1)} and T2 = {(i,j), (i+1,j+1), (i,j+1)}.  Boundary nodes
carry homogeneous Dirichlet data (Sec. 6: u = 0 on all four sides) and are eliminated.
Element matrices are the textbook P1 ones written from vertex coordinates:
  K_e = area * grad(phi) grad(phi)^T   (scaled by the element's coefficient)
  M_e = area / 12 * [[2,1,1],[1,2,1],[1,1,2]]   (consistent mass)
Coefficients are evaluated at element centroids (one-point rule, exact for P1
gradients with an elementwise-constant coefficient).
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import field, kl


def node_id(i: int, j: int, N: int) -> int:
    return j * (N + 1) + i


def elements(N: int):
    """Returns (tri, centroids): tri (2N^2, 3) global node ids; element index
    e = 2 (j N + i) + t, t = 0 for T1 and 1 for T2."""
    tri = np.zeros((2 * N * N, 3), dtype=np.int64)
    cen = np.zeros((2 * N * N, 2))
    h = 1.0 / N
    for j in range(N):
        for i in range(N):
            e = 2 * (j * N + i)
            tri[e] = (node_id(i, j, N), node_id(i + 1, j, N), node_id(i + 1, j + 1, N))
            tri[e + 1] = (node_id(i, j, N), node_id(i + 1, j + 1, N), node_id(i, j + 1, N))
            cen[e] = ((i + 2.0 / 3.0) * h, (j + 1.0 / 3.0) * h)
            cen[e + 1] = ((i + 1.0 / 3.0) * h, (j + 2.0 / 3.0) * h)
    return tri, cen


def node_xy(N: int):
    h = 1.0 / N
    idx = np.arange((N + 1) ** 2)
    return (idx % (N + 1)) * h, (idx // (N + 1)) * h


def element_matrices(xy: np.ndarray):
    """P1 stiffness (unit coefficient) and consistent mass for one triangle."""
    (x1, y1), (x2, y2), (x3, y3) = xy
    area = 0.5 * abs((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1))
    # gradients of barycentric functions: grad(phi_a) = (y_b - y_c, x_c - x_b) / (2 area)
    b = np.array([y2 - y3, y3 - y1, y1 - y2])
    c = np.array([x3 - x2, x1 - x3, x2 - x1])
    K = (np.outer(b, b) + np.outer(c, c)) / (4 * area)
    Mm = area / 12.0 * np.array([[2.0, 1, 1], [1, 2, 1], [1, 1, 2]])
    return K, Mm


def element_coefficients(prob) -> np.ndarray:
    """c[alpha, e]: PCE coefficients of c_s = exp(g) at element centroids (Sec. 4)."""
    _, cen = elements(prob.N)
    gn = kl.kl_fields(prob.M, prob.sigma, prob.bx, prob.by, cen[:, 0], cen[:, 1])
    return field.lognormal_pce(gn, prob.g0, prob.p_in)


def assemble(N: int, coef: np.ndarray, elem_mask=None):
    """Assemble over all (or the masked) elements on ALL (N+1)^2 nodes.

    coef: (P_in, n_elem).  Returns (M, [K_0 .. K_{P_in-1}]) as CSR matrices where
    K_i = sum_e coef[i, e] K_e (the PCE coefficient matrices of Sec. 4, Eq. stok)."""
    tri, _ = elements(N)
    X, Y = node_xy(N)
    nn = (N + 1) ** 2
    eids = np.arange(tri.shape[0]) if elem_mask is None else np.nonzero(elem_mask)[0]
    Kloc = np.zeros((eids.size, 3, 3))
    Mloc = np.zeros((eids.size, 3, 3))
    for n, e in enumerate(eids):
        v = tri[e]
        Kloc[n], Mloc[n] = element_matrices(np.stack([X[v], Y[v]], axis=1))
    v = tri[eids]
    rows = np.repeat(v, 3, axis=1).ravel()          # v[a] repeated for each b
    cols = np.tile(v, (1, 3)).ravel()               # v[b]
    Mmat = sp.csr_matrix((Mloc.ravel(), (rows, cols)), shape=(nn, nn))
    Ks = []
    for i in range(coef.shape[0]):
        vals = (Kloc * coef[i, eids][:, None, None]).ravel()
        Ks.append(sp.csr_matrix((vals, (rows, cols)), shape=(nn, nn)))
    return Mmat, Ks


def free_nodes(N: int) -> np.ndarray:
    """Global ids of the interior (non-Dirichlet) nodes, in (j, i) row-major order."""
    return np.array([node_id(i, j, N) for j in range(1, N) for i in range(1, N)], dtype=np.int64)


def p1_values(N: int, x: float, y: float) -> Dict[int, float]:
    """Values of the P1 basis functions at the point (x, y): {global node: phi}."""
    h = 1.0 / N
    i = min(int(math.floor(x / h)), N - 1)
    j = min(int(math.floor(y / h)), N - 1)
    fx = x / h - i
    fy = y / h - j
    if fy <= fx:  # T1: (i,j), (i+1,j), (i+1,j+1)
        w = {node_id(i, j, N): 1.0 - fx, node_id(i + 1, j, N): fx - fy, node_id(i + 1, j + 1, N): fy}
    else:  # T2: (i,j), (i+1,j+1), (i,j+1)
        w = {node_id(i, j, N): 1.0 - fy, node_id(i + 1, j + 1, N): fx, node_id(i, j + 1, N): fy - fx}
    return {k: v for k, v in w.items() if v != 0.0}


def ricker(t: float, freq: float) -> float:
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - 1/f.
    Reading: the paper has no source term of this kind; the workloads add it."""
    tau = t - 1.0 / freq
    a = (math.pi * freq * tau) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def point_load(N: int, src, t: float) -> np.ndarray:
    """Deterministic nodal load f(t) on all nodes for a point source r(t) delta(x - x_s):
    F_a = amp r(t) phi_a(x_s)."""
    f = np.zeros((N + 1) ** 2)
    if src.kind == 2:
        r = src.amp * ricker(t, src.freq)
        for a, v in p1_values(N, src.x0, src.y0).items():
            f[a] += r * v
    return f


def initial_displacement(N: int, src) -> np.ndarray:
    """Nodal interpolation of the Gaussian pulse u0 = amp exp(-r^2 / width^2) (Sec. 6.2,
    Eq. initial_2Dwave with alpha = width^2, beta = amp)."""
    X, Y = node_xy(N)
    if src.kind == 1:
        return src.amp * np.exp(-((X - src.x0) ** 2 + (Y - src.y0) ** 2) / src.width ** 2)
    return np.zeros((N + 1) ** 2)
