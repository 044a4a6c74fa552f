"""Seeded unstructured meshes of the unit square and element partitions: the inputs of the
general-partition path, shared by the oracle, the tests and bench.py.  Mesh generation and
partitioning only (vertex coordinates, triangles, Dirichlet flags, subdomain ids); none of the
solver's arithmetic (no classes, no assembly, no solves).

The paper's meshes (1563 to 53263 vertices) and its partitioner are not available (Sec. 6), so:
  * `delaunay_square(n, jitter, seed)`: n + 1 boundary vertices per side, an (n - 1)^2 interior grid
    jittered by up to `jitter` cells with SplitMix64 draws, Delaunay triangulation (slivers of
    co-circular boundary points dropped).  n = 192 gives 37249 vertices, the size of the paper's
    37267-vertex mesh of the scaling-with-random-variables study (Sec. 6.4).
  * `rcb_partition(xy, tri, nparts)`: recursive coordinate bisection of the triangles by centroid,
    across the longer extent, at the count-weighted median; any number of subdomains.
"""
from __future__ import annotations

import numpy as np

from . import uniform_samples


def _on_boundary(xy: np.ndarray) -> np.ndarray:
    eps = 1e-12
    return (xy[:, 0] < eps) | (xy[:, 0] > 1 - eps) | (xy[:, 1] < eps) | (xy[:, 1] > 1 - eps)


def delaunay_square(n: int, jitter: float = 0.3, seed: int = 7):
    """(xy (nv, 2), tri (ne, 3), boundary (nv,) bool) of the seeded mesh described above."""
    from scipy.spatial import Delaunay
    h = 1.0 / n
    pts = []
    for k in range(n + 1):  # boundary, every vertex once
        pts += [(k * h, 0.0), (k * h, 1.0)]
    for k in range(1, n):
        pts += [(0.0, k * h), (1.0, k * h)]
    u = uniform_samples(2 * (n - 1) ** 2, seed)
    q = 0
    for j in range(1, n):
        for i in range(1, n):
            dx = (2.0 * u[q] - 1.0) * jitter * h
            dy = (2.0 * u[q + 1] - 1.0) * jitter * h
            q += 2
            pts.append((i * h + dx, j * h + dy))
    xy = np.array(pts)
    tri = Delaunay(xy).simplices
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))
    tri = tri[area > 1e-12 * h * h]
    return xy, tri, _on_boundary(xy)


def rcb_partition(xy: np.ndarray, tri: np.ndarray, nparts: int) -> np.ndarray:
    """Triangle -> subdomain id by recursive coordinate bisection of the centroids."""
    cen = (xy[tri[:, 0]] + xy[tri[:, 1]] + xy[tri[:, 2]]) / 3.0
    part = np.zeros(tri.shape[0], dtype=np.int64)

    def split(ids: np.ndarray, k: int, first: int):
        if k == 1:
            part[ids] = first
            return
        c = cen[ids]
        ax = 0 if np.ptp(c[:, 0]) >= np.ptp(c[:, 1]) else 1
        order = ids[np.lexsort((c[:, 1 - ax], c[:, ax]))]
        k0 = k // 2
        n0 = (ids.size * k0) // k
        split(order[:n0], k0, first)
        split(order[n0:], k - k0, first + k0)

    split(np.arange(tri.shape[0]), nparts, 0)
    return part
