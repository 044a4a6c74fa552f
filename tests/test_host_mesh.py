"""The library's host set-up for unstructured meshes and general partitions (csrc/sg_host.cpp,
build_mesh_problem; compiled here with g++ into a small dump program, no GPU) against the oracle's
general-partition path (oracle/umesh.py, written independently): vertex classes with the corner
reading of Sec. 3, multiplicities, local vertices, the edges of every subdomain with their stiffness
weights per PCE input mode (minus the oracle's local K_i entries), triangle areas and KL eigenvalues."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import sg_workloads as w
from oracle import kl, umesh

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("hostmesh") / "mesh_dump"
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", str(out), os.path.join(HERE, "helpers", "mesh_dump.cpp"),
                    os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_host.cpp"), "-lpthread"],
                   check=True, capture_output=True)
    return str(out)


def dump(exe, tmp_path, mesh, part, prob):
    path = tmp_path / "mesh.txt"
    with open(path, "w") as f:
        f.write(f"{mesh.nn} {mesh.tri.shape[0]} {prob.M} {float(prob.sigma):.17g} {float(prob.bx):.17g} "
                f"{float(prob.by):.17g} {float(prob.g0):.17g} {prob.p} {prob.p_in}\n")
        for (x, y), d in zip(mesh.xy, mesh.boundary):
            f.write(f"{float(x):.17g} {float(y):.17g} {int(d)}\n")
        for t, s in zip(mesh.tri, part):
            f.write(f"{t[0]} {t[1]} {t[2]} {s}\n")
    txt = subprocess.run([exe, str(path)], check=True, capture_output=True, text=True).stdout
    out = {"sub": {}}
    for line in txt.splitlines():
        name, *vals = line.split()
        if name in ("verts", "edges", "weights", "areas"):
            s = int(vals[0])
            out["sub"].setdefault(s, {})[name] = np.array([float(v) for v in vals[1:]])
        else:
            out[name] = np.array([float(v) for v in vals])
    return out


def cases():
    out = []
    m = umesh.delaunay_mesh(12, 0.3, 11)
    out += [("delaunay12_rcb3", m, umesh.rcb_partition(m, 3)), ("delaunay12_rcb5", m, umesh.rcb_partition(m, 5))]
    m = umesh.delaunay_mesh(9, 0.35, 4)
    out.append(("delaunay9_rcb6", m, umesh.rcb_partition(m, 6)))
    N = 4
    m = umesh.structured_mesh(N)
    cx, cy = (m.cen[:, 0] * N).astype(int), (m.cen[:, 1] * N).astype(int)
    out.append(("tjunction", m, np.where(cx < 2, 0, np.where(cy < 2, 1, 2))))
    out.append(("pinch", m, ((cx >= 2).astype(int) + (cy >= 2).astype(int)) % 2))
    N = 6
    m = umesh.structured_mesh(N)
    cx, cy = (m.cen[:, 0] * N).astype(int), (m.cen[:, 1] * N).astype(int)
    out.append(("island", m, ((cx >= 2) & (cx < 4) & (cy >= 2) & (cy < 4)).astype(int)))
    return out


CASES = cases()


@pytest.mark.parametrize("name,mesh,part", CASES, ids=[c[0] for c in CASES])
def test_mesh_setup_matches_oracle(dump_exe, tmp_path, name, mesh, part):
    prob = w.config("small").replace(M=3, p=2, p_in=2, sigma=0.3, bx=0.4, by=0.6)
    up = umesh.UPartition(mesh, part)
    t = dump(dump_exe, tmp_path, mesh, part, prob)
    nv, ne, nsub, P, PI, n_free, nG, nC = t["sizes"].astype(int)
    assert (nv, ne, nsub) == (mesh.nn, mesh.tri.shape[0], up.nsub)
    assert (n_free, nG, nC) == (up.free.size, up.iface.size, up.corner.size)
    # vertex classes and multiplicities
    cls = np.zeros(mesh.nn, dtype=int)
    cls[up.free] = 1
    cls[up.iface] = 2
    cls[up.corner] = 3
    assert np.array_equal(t["vclass"].astype(int), cls)
    assert np.array_equal(t["vmult"].astype(int), [len(s) for s in up.node_subs])
    # KL eigenvalues: the analytic top-M products, in the oracle's order
    lam = [l for l, _, _ in kl.kl_modes(prob.M, prob.bx, prob.by)]
    assert np.allclose(t["kl_lambda"], lam, rtol=1e-12, atol=0)
    coef = up.element_coefficients(prob)
    tot_area = 0.0
    for s in range(nsub):
        d = t["sub"][s]
        verts = d["verts"].astype(int)
        sub = up.subs[s]
        # local vertices: the oracle's free vertices plus the Dirichlet ones, classes in order
        assert set(verts[cls[verts] > 0].tolist()) == set(sub["nodes"].tolist())
        order = np.where(cls[verts] == 0, 4, cls[verts])
        assert np.all(np.diff(order) >= 0)
        assert set(verts.tolist()) == set(np.unique(mesh.tri[part == s]).tolist())
        # edges: exactly the triangle edges of the subdomain; weights = -K_i[a, b] of its elements
        e = d["edges"].astype(int).reshape(-1, 2)
        tri_edges = {tuple(sorted((int(a), int(b)))) for tt in mesh.tri[part == s]
                     for a, b in ((tt[0], tt[1]), (tt[1], tt[2]), (tt[2], tt[0]))}
        assert {tuple(sorted(x)) for x in e.tolist()} == tri_edges and len(e) == len(tri_edges)
        W = d["weights"].reshape(len(e), PI)
        _, Ks = up.assemble(coef, sub["elem_mask"])
        for i in range(PI):
            Kd = Ks[i].toarray()
            ref = -Kd[e[:, 0], e[:, 1]]
            assert np.abs(W[:, i] - ref).max() <= 1e-12 * max(np.abs(Kd).max(), 1e-300)
        # areas, element by element
        assert np.allclose(d["areas"], mesh.area[part == s], rtol=1e-13, atol=0)
        tot_area += d["areas"].sum()
    assert abs(tot_area - 1.0) < 1e-12


def test_mesh_setup_rejects_bad_partitions(dump_exe, tmp_path):
    """Subdomain ids must be 0 .. nsub - 1 with every id used."""
    m = umesh.delaunay_mesh(6, 0.3, 5)
    part = umesh.rcb_partition(m, 3)
    part = np.where(part == 1, 2, part)   # id 1 unused
    prob = w.config("small")
    with pytest.raises(subprocess.CalledProcessError) as e:
        dump(dump_exe, tmp_path, m, part, prob)
    assert e.value.returncode == 1 and "subdomain ids" in e.value.stderr
