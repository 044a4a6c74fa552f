"""Unstructured triangle meshes and general partitions for the SG-DD oracle (test infrastructure;
the paper's experiments use unstructured meshes of the unit square split into subdomains, Sec. 6,
with corners defined in Sec. 3).

* `Mesh`: vertex coordinates, counter-clockwise triangles, Dirichlet (boundary) vertices.
  `structured_mesh(N)` is the structured grid of `fem` with the same numbering (the pin that ties
  this module to the structured oracle); `delaunay_mesh(n, jitter, seed)` wraps the seeded
  unstructured mesh of the shared input generator (sg_workloads.meshes): n + 1 boundary vertices
  per side, an (n - 1)^2 interior grid jittered by up to `jitter` cells (SplitMix64 draws),
  Delaunay triangulation.
* `rcb_partition(mesh, nparts)`: recursive coordinate bisection of the elements (by centroid,
  across the longer extent, at the count-weighted median), for any number of subdomains, from the
  same input generator.
* `UPartition`: node classes and restriction maps of an element partition, with the attributes of
  `dd.Partition`.  Interface nodes are free vertices of elements of two or more subdomains.
  Corners (reading of Sec. 3: nodes shared by more than two subdomains, plus the end nodes of
  interface edges): free interface vertices in three or more subdomains, and free interface
  vertices in exactly two subdomains A, B that do not have exactly two incident A|B interface edges
  (an edge whose two triangles lie in A and B); an interface curve that reaches the boundary ends at
  a Dirichlet vertex, which is eliminated.  D_s is the counting partition of unity.
* `USGProblem`: the global SG system of a workload on a mesh (free vertices only), with the Ricker
  point source located by barycentric coordinates.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np
import scipy.sparse as sp

from . import fem, field, kl, pce
from .sg import SGOperators

import sg_workloads as w
from sg_workloads import meshes


class Mesh:
    def __init__(self, xy: np.ndarray, tri: np.ndarray, boundary: np.ndarray):
        self.xy = np.asarray(xy, dtype=float)
        tri = np.asarray(tri, dtype=np.int64).copy()
        a = self.xy[tri[:, 0]]
        b = self.xy[tri[:, 1]]
        c = self.xy[tri[:, 2]]
        area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])
        flip = area2 < 0
        tri[flip] = tri[flip][:, [0, 2, 1]]
        self.tri = tri
        self.area = 0.5 * np.abs(area2)
        self.cen = (a + b + c) / 3.0
        self.boundary = np.asarray(boundary, dtype=bool)
        self.nn = self.xy.shape[0]

    @property
    def free(self) -> np.ndarray:
        return np.nonzero(~self.boundary)[0].astype(np.int64)

    def edges(self) -> Dict[tuple, List[int]]:
        """{(u, v) with u < v: [elements containing the edge]}."""
        out: Dict[tuple, List[int]] = {}
        for e, (p, q, r) in enumerate(self.tri):
            for u, v in ((p, q), (q, r), (r, p)):
                key = (min(u, v), max(u, v))
                out.setdefault(key, []).append(e)
        return out


def _on_boundary(xy: np.ndarray) -> np.ndarray:
    eps = 1e-12
    return (xy[:, 0] < eps) | (xy[:, 0] > 1 - eps) | (xy[:, 1] < eps) | (xy[:, 1] > 1 - eps)


def structured_mesh(N: int) -> Mesh:
    """The structured grid of `fem` (same vertex and element numbering)."""
    tri, _ = fem.elements(N)
    X, Y = fem.node_xy(N)
    xy = np.stack([X, Y], axis=1)
    return Mesh(xy, tri, _on_boundary(xy))


def delaunay_mesh(n: int, jitter: float = 0.3, seed: int = 7) -> Mesh:
    """Seeded unstructured mesh of the unit square (the shared input generator
    sg_workloads.meshes.delaunay_square; see the module docstring)."""
    xy, tri, boundary = meshes.delaunay_square(n, jitter, seed)
    return Mesh(xy, tri, boundary)


def rcb_partition(mesh: Mesh, nparts: int) -> np.ndarray:
    """Element -> subdomain by recursive coordinate bisection of the centroids (the shared input
    generator sg_workloads.meshes.rcb_partition on this mesh's triangles)."""
    return meshes.rcb_partition(mesh.xy, mesh.tri, nparts)


class UPartition:
    """Node classes and restriction maps of an element partition of a mesh (attributes as
    dd.Partition)."""

    def __init__(self, mesh: Mesh, part: np.ndarray):
        self.mesh = mesh
        self.part = np.asarray(part, dtype=np.int64)
        ns = int(self.part.max()) + 1
        self.nsub = ns
        node_subs: List[set] = [set() for _ in range(mesh.nn)]
        for e, v in enumerate(mesh.tri):
            for a in v:
                node_subs[a].add(int(self.part[e]))
        self.node_subs = node_subs
        self.free = mesh.free
        self.free_index = {int(g): k for k, g in enumerate(self.free)}
        # interface edges per node: {node: {pair: count}}
        iedge: Dict[int, Dict[tuple, int]] = {}
        for (u, v), els in mesh.edges().items():
            if len(els) == 2:
                pa, pb = int(self.part[els[0]]), int(self.part[els[1]])
                if pa != pb:
                    pair = (min(pa, pb), max(pa, pb))
                    for x in (u, v):
                        d = iedge.setdefault(int(x), {})
                        d[pair] = d.get(pair, 0) + 1
        iface, corner = [], []
        for g in self.free:
            g = int(g)
            s = node_subs[g]
            if len(s) < 2:
                continue
            iface.append(g)
            if len(s) >= 3:
                corner.append(g)
            else:
                pair = tuple(sorted(s))
                if iedge.get(g, {}).get(pair, 0) != 2:
                    corner.append(g)
        self.iface = np.array(iface, dtype=np.int64)
        self.iface_index = {int(g): k for k, g in enumerate(self.iface)}
        self.corner = np.array(corner, dtype=np.int64)
        self.corner_index = {int(g): k for k, g in enumerate(self.corner)}
        self.mult = np.array([len(node_subs[int(g)]) for g in self.iface], dtype=float)
        self.subs = []
        for si in range(ns):
            em = self.part == si
            nodes = np.unique(mesh.tri[em].ravel())
            loc = np.array([g for g in nodes if int(g) in self.free_index], dtype=np.int64)
            cls = np.array(["c" if int(g) in self.corner_index else "r" if int(g) in self.iface_index else "i"
                            for g in loc])
            self.subs.append({"nodes": loc, "cls": cls,
                              "gamma": np.array([g for g in loc if int(g) in self.iface_index], dtype=np.int64),
                              "elem_mask": em})

    def assemble(self, coef: np.ndarray, elem_mask=None):
        return assemble(self.mesh, coef, elem_mask)

    def element_coefficients(self, prob) -> np.ndarray:
        return element_coefficients(self.mesh, prob)


def assemble(mesh: Mesh, coef: np.ndarray, elem_mask=None):
    """M and K_i = sum_e coef[i, e] K_e over all (or the masked) elements, on all vertices."""
    eids = np.arange(mesh.tri.shape[0]) if elem_mask is None else np.nonzero(elem_mask)[0]
    Kloc = np.zeros((eids.size, 3, 3))
    Mloc = np.zeros((eids.size, 3, 3))
    for n, e in enumerate(eids):
        Kloc[n], Mloc[n] = fem.element_matrices(mesh.xy[mesh.tri[e]])
    v = mesh.tri[eids]
    rows = np.repeat(v, 3, axis=1).ravel()
    cols = np.tile(v, (1, 3)).ravel()
    nn = mesh.nn
    Mmat = sp.csr_matrix((Mloc.ravel(), (rows, cols)), shape=(nn, nn))
    Ks = []
    for i in range(coef.shape[0]):
        Ks.append(sp.csr_matrix(((Kloc * coef[i, eids][:, None, None]).ravel(), (rows, cols)), shape=(nn, nn)))
    return Mmat, Ks


def element_coefficients(mesh: Mesh, prob) -> np.ndarray:
    """PCE coefficients of c_s = exp(g) at the element centroids (one-point rule, Sec. 4)."""
    gn = kl.kl_fields(prob.M, prob.sigma, prob.bx, prob.by, mesh.cen[:, 0], mesh.cen[:, 1])
    return field.lognormal_pce(gn, prob.g0, prob.p_in)


def p1_values(mesh: Mesh, x: float, y: float) -> Dict[int, float]:
    """P1 basis values at (x, y): barycentric coordinates in the first element that contains it."""
    a, b, c = mesh.xy[mesh.tri[:, 0]], mesh.xy[mesh.tri[:, 1]], mesh.xy[mesh.tri[:, 2]]
    det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])
    l1 = ((x - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (y - a[:, 1])) / det
    l2 = ((b[:, 0] - a[:, 0]) * (y - a[:, 1]) - (x - a[:, 0]) * (b[:, 1] - a[:, 1])) / det
    l0 = 1.0 - l1 - l2
    inside = np.nonzero((l0 >= -1e-12) & (l1 >= -1e-12) & (l2 >= -1e-12))[0]
    e = int(inside[0])
    v = mesh.tri[e]
    return {int(v[0]): float(l0[e]), int(v[1]): float(l1[e]), int(v[2]): float(l2[e])}


class USGProblem:
    """Global SG system of a workload on a mesh (free vertices only); the analogue of
    sg.SGProblem with the structured grid replaced by `mesh`."""

    def __init__(self, mesh: Mesh, prob, coef=None):
        self.prob = prob
        self.mesh = mesh
        self.coef = element_coefficients(mesh, prob) if coef is None else coef
        Mfull, Kfull = assemble(mesh, self.coef)
        f = self.free = mesh.free
        self.M = Mfull[f][:, f].tocsr()
        self.Ks = [K[f][:, f].tocsr() for K in Kfull]
        self.G = pce.triple_products(prob.M, prob.p_in, prob.p)
        self.P = self.G.shape[1]
        self.ops = SGOperators(self.M, self.Ks, self.G, prob.alpha0, prob.alpha1, prob.dt)
        src = prob.source
        self._src = p1_values(mesh, src.x0, src.y0) if src.kind == 2 else {}

    def load(self, t: float) -> np.ndarray:
        fn = np.zeros(self.mesh.nn)
        src = self.prob.source
        if src.kind == 2:
            r = src.amp * fem.ricker(t, src.freq)
            for a, v in self._src.items():
                fn[a] += r * v
        F = np.zeros((self.free.size, self.P))
        F[:, 0] = fn[self.free]
        return F.ravel()

    def initial_state(self):
        n = self.free.size
        U0 = np.zeros((n, self.P))
        src = self.prob.source
        if src.kind == 1:
            xy = self.mesh.xy[self.free]
            U0[:, 0] = src.amp * np.exp(-((xy[:, 0] - src.x0) ** 2 + (xy[:, 1] - src.y0) ** 2) / src.width ** 2)
        U0 = U0.ravel()
        V0 = np.zeros_like(U0)
        A0 = self.ops.initial_acceleration(self.load(0.0), U0, V0)
        return U0, V0, A0
