"""Pins of the oracle's unstructured-mesh path (oracle/umesh.py): meshes, general partitions, corner
detection (Sec. 3) and the SG-DD solve on them.

The structured grid run through the unstructured path must reproduce the structured oracle (node
classes and DD-PCG iterates), which ties the general code to the pinned structured one; on
unstructured meshes the DD-PCG at tol 1e-13 must equal the direct solve of the global SG system, the
matrix-free Schur complement its dense form, and the preconditioner stay SPD.  Mesh pins: areas sum
to the unit square, the Euler relation of a triangulated disk, the P1 patch test (linear functions
are discretely harmonic), the mass of the constant."""
import numpy as np
import pytest

import sg_workloads as w
from oracle import dd, sg, umesh


def block_partition(mesh, N, s):
    H = N // s
    ci = np.minimum((mesh.cen[:, 0] * N).astype(int) // H, s - 1)
    cj = np.minimum((mesh.cen[:, 1] * N).astype(int) // H, s - 1)
    return cj * s + ci


@pytest.mark.parametrize("N,s", [(24, 3), (16, 4)])
def test_structured_grid_through_the_general_partition(N, s):
    prob = w.config("small").replace(N=N, s=s, dt=w.cfl_dt(N))
    m = umesh.structured_mesh(N)
    up = umesh.UPartition(m, block_partition(m, N, s))
    p0 = dd.Partition(N, s)
    assert np.array_equal(np.sort(up.free), np.sort(p0.free))
    assert set(up.iface.tolist()) == set(p0.iface.tolist())
    assert set(up.corner.tolist()) == set(p0.corner.tolist())
    assert up.corner.size == (s - 1) ** 2
    m0 = {int(g): v for g, v in zip(p0.iface, p0.mult)}
    assert all(m0[int(g)] == v for g, v in zip(up.iface, up.mult))
    for a, b in zip(p0.subs, up.subs):
        assert set(a["nodes"].tolist()) == set(b["nodes"].tolist())
    sgp = sg.SGProblem(prob)
    U0, _, _, it0 = dd.run_dd(sgp, dd.DDSolver(prob), 3, tol=1e-13)
    U1, _, _, it1 = dd.run_dd(sgp, dd.DDSolver(prob, partition=up), 3, tol=1e-13)
    assert np.linalg.norm(U1 - U0) <= 1e-13 * np.linalg.norm(U0)
    assert [i for i, _ in it0] == [i for i, _ in it1]


@pytest.mark.parametrize("n,jitter,seed", [(8, 0.3, 1), (16, 0.35, 7)])
def test_delaunay_mesh(n, jitter, seed):
    m = umesh.delaunay_mesh(n, jitter, seed)
    assert m.nn == (n + 1) ** 2
    assert np.all(m.area > 0)
    assert abs(m.area.sum() - 1.0) < 1e-12
    E = len(m.edges())
    assert m.nn - E + m.tri.shape[0] == 1          # Euler relation of a triangulated disk
    assert m.boundary.sum() == 4 * n
    # counter-clockwise orientation
    a, b, c = m.xy[m.tri[:, 0]], m.xy[m.tri[:, 1]], m.xy[m.tri[:, 2]]
    assert np.all((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]) > 0)
    M, Ks = umesh.assemble(m, np.ones((1, m.tri.shape[0])))
    one = np.ones(m.nn)
    assert abs(one @ (M @ one) - 1.0) < 1e-12        # mass of the constant = area
    K = Ks[0]
    assert np.abs(K @ one).max() < 1e-12             # constants are in the kernel
    for lin in (m.xy[:, 0], m.xy[:, 1], 0.3 * m.xy[:, 0] - 1.7 * m.xy[:, 1] + 0.2):
        r = K @ lin                                   # patch test: linear functions are discretely harmonic
        assert np.abs(r[~m.boundary]).max() < 1e-11


@pytest.mark.parametrize("nparts", [2, 3, 5, 6])
def test_rcb_partition_is_balanced(nparts):
    m = umesh.delaunay_mesh(16, 0.3, 3)
    part = umesh.rcb_partition(m, nparts)
    cnt = np.bincount(part, minlength=nparts)
    assert cnt.size == nparts and cnt.sum() == m.tri.shape[0]
    assert cnt.max() - cnt.min() <= 1


def test_corner_detection():
    """Sec. 3 reading: corners are free interface vertices in three or more subdomains, and end
    vertices of interface curves (a free vertex of two subdomains without exactly two interface
    edges between them)."""
    N = 4
    m = umesh.structured_mesh(N)
    cx, cy = (m.cen[:, 0] * N).astype(int), (m.cen[:, 1] * N).astype(int)
    node = lambda i, j: j * (N + 1) + i
    # T-junction: left half, right-bottom, right-top -> the junction vertex only
    part = np.where(cx < 2, 0, np.where(cy < 2, 1, 2))
    up = umesh.UPartition(m, part)
    assert up.corner.tolist() == [node(2, 2)]
    # two subdomains in a 2 x 2 checkerboard of blocks: the centre is pinched (four interface edges)
    part = ((cx >= 2).astype(int) + (cy >= 2).astype(int)) % 2
    up = umesh.UPartition(m, part)
    assert up.corner.tolist() == [node(2, 2)]
    assert set(up.iface.tolist()) == {node(2, 1), node(2, 3), node(1, 2), node(3, 2), node(2, 2)}
    # an island inside another subdomain: a closed interface curve, no corners
    N = 6
    m = umesh.structured_mesh(N)
    cx, cy = (m.cen[:, 0] * N).astype(int), (m.cen[:, 1] * N).astype(int)
    part = ((cx >= 2) & (cx < 4) & (cy >= 2) & (cy < 4)).astype(int)
    up = umesh.UPartition(m, part)
    assert up.corner.size == 0 and up.iface.size == 8


@pytest.mark.parametrize("nparts", [3, 5])
def test_unstructured_dd_pcg_matches_direct(nparts):
    prob = w.config("small").replace(name="u12", N=12, s=2, dt=0.02)
    m = umesh.delaunay_mesh(12, 0.3, 11)
    up = umesh.UPartition(m, umesh.rcb_partition(m, nparts))
    usg = umesh.USGProblem(m, prob)
    Ud, _, _, it = dd.run_dd(usg, dd.DDSolver(prob, partition=up), 3, tol=1e-13)
    Ur, _, _ = sg.run_direct(usg, 3)
    assert np.linalg.norm(Ud - Ur) <= 1e-10 * np.linalg.norm(Ur)
    assert all(rel <= 1e-13 for _, rel in it)


def test_unstructured_explicit_operators():
    """Matrix-free Schur complement and two-level preconditioner equal their dense forms (Eqs.
    Sto_Schur, Fcc_2, NNCP2) on an unstructured 3-subdomain partition; both are SPD."""
    prob = w.config("tiny").replace(name="u6", N=6, s=2)
    m = umesh.delaunay_mesh(6, 0.3, 5)
    up = umesh.UPartition(m, umesh.rcb_partition(m, 3))
    d = dd.DDSolver(prob, explicit=True, partition=up)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(d.nG * d.P)
    Sx = d.schur(x)
    assert np.abs(Sx - d.S_explicit @ x).max() < 1e-10 * np.abs(Sx).max()
    z = d.precond(x)
    assert np.abs(z - d.Minv_explicit @ x).max() < 1e-10 * np.abs(z).max()
    for A in (d.S_explicit, d.Minv_explicit):
        assert np.allclose(A, A.T, atol=1e-10 * np.abs(A).max())
        assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_point_source_basis_values():
    """The point source's P1 basis values (barycentric coordinates) reproduce linear functions at
    any point and sum to one; on the structured grid the global load equals the structured
    oracle's."""
    m = umesh.delaunay_mesh(10, 0.3, 2)
    rng = np.random.default_rng(4)
    for x, y in rng.uniform(0.0, 1.0, (25, 2)):
        phi = umesh.p1_values(m, x, y)
        assert abs(sum(phi.values()) - 1.0) < 1e-12
        for f in (lambda X, Y: X, lambda X, Y: Y, lambda X, Y: 0.7 * X - 0.2 * Y + 0.5):
            val = sum(v * f(*m.xy[a]) for a, v in phi.items())
            assert abs(val - f(x, y)) < 1e-12
    prob = w.config("small")
    ms = umesh.structured_mesh(prob.N)
    a, b = umesh.USGProblem(ms, prob), sg.SGProblem(prob)
    for t in (0.05, 0.1, 0.13):
        assert np.abs(a.load(t) - b.load(t)).max() < 1e-14


def test_pulse_initial_state_on_the_structured_grid():
    """The Gaussian-pulse initial state (U_0 interpolated, V_0 = 0, consistent A_0) of the mesh-based
    problem equals the structured oracle's on the structured grid."""
    prob = w.config("tiny")
    a = umesh.USGProblem(umesh.structured_mesh(prob.N), prob).initial_state()
    b = sg.SGProblem(prob).initial_state()
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)


@pytest.mark.parametrize("pc", ["nn1", "lumped"])
def test_unstructured_one_level_preconditioners(pc):
    """The comparison preconditioners of Sec. 6.1 on a general partition: DD-PCG at tol 1e-13 equals
    the direct SG solve; the two-level preconditioner needs no more iterations than the one-level
    NN (with four subdomains and few corners its coarse space adds little) and fewer than lumped."""
    prob = w.config("small").replace(name="u10", N=10, s=2, dt=0.02)
    m = umesh.delaunay_mesh(10, 0.3, 13)
    up = umesh.UPartition(m, umesh.rcb_partition(m, 4))
    usg = umesh.USGProblem(m, prob)
    Ud, _, _, it = dd.run_dd(usg, dd.DDSolver(prob, partition=up, precond=pc), 2, tol=1e-13)
    Ur, _, _ = sg.run_direct(usg, 2)
    assert np.linalg.norm(Ud - Ur) <= 1e-10 * np.linalg.norm(Ur)
    _, _, _, it2 = dd.run_dd(usg, dd.DDSolver(prob, partition=up), 2, tol=1e-13)
    if pc == "nn1":
        assert sum(i for i, _ in it2) <= sum(i for i, _ in it)
    else:
        assert sum(i for i, _ in it2) < sum(i for i, _ in it)
