"""The library's host set-up for unstructured meshes and general partitions (csrc/sg_host.cpp,
build_mesh_problem, mesh_to_problem, mesh_mean_inverse; compiled here with g++ into a small dump
program, no GPU) against the oracle's general-partition path (oracle/umesh.py, written
independently): vertex classes with the corner reading of Sec. 3, multiplicities, local vertices, the
edges of every subdomain with their stiffness weights per PCE input mode (minus the oracle's local K_i
entries), triangle areas and KL eigenvalues; then the device layout the solver runs on: the sparse
rows of every subdomain's mass and stiffness matrices (equal to the oracle's local matrices), the
interface and corner maps, the output maps, the initial pulse, the point load (the oracle's P1 values
split over the owning subdomains), the triple-product table and the inverses of the mean operator."""
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


def dump(exe, tmp_path, mesh, part, prob, layout=None):
    path = tmp_path / "mesh.txt"
    with open(path, "w") as f:
        f.write(f"{mesh.nn} {mesh.tri.shape[0]} {prob.M} {float(prob.sigma):.17g} {float(prob.bx):.17g} "
                f"{float(prob.by):.17g} {float(prob.g0):.17g} {prob.p} {prob.p_in}\n")
        for (x, y), d in zip(mesh.xy, mesh.boundary):
            f.write(f"{float(x):.17g} {float(y):.17g} {int(d)}\n")
        for t, s in zip(mesh.tri, part):
            f.write(f"{t[0]} {t[1]} {t[2]} {s}\n")
    args = [exe, str(path)]
    if layout is not None:
        lpath = tmp_path / "layout.txt"
        lpath.write_text(" ".join(f"{float(v):.17g}" if not isinstance(v, int) else str(v) for v in layout) + "\n")
        args.append(str(lpath))
    txt = subprocess.run(args, check=True, capture_output=True, text=True).stdout
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


LAYOUT_CASES = [c for c in CASES if c[0] in ("delaunay12_rcb5", "delaunay9_rcb6", "tjunction", "pinch", "island")]


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("name,mesh,part", LAYOUT_CASES, ids=[c[0] for c in LAYOUT_CASES])
def test_mesh_device_layout_matches_oracle(dump_exe, tmp_path, name, mesh, part, kind):
    prob = w.config("small").replace(M=3, p=2, p_in=2, sigma=0.3, bx=0.4, by=0.6)
    src = w.Source(kind, 0.37, 0.61, 0.15, 8.0, 1.3)
    dt, a0, a1 = 0.02, 0.3, 0.002
    zeta, gamma = 0.25, 0.5
    am = 1.0 / (zeta * dt * dt) + a0 * gamma / (zeta * dt)
    bk = 1.0 + a1 * gamma / (zeta * dt)
    up = umesh.UPartition(mesh, part)
    t = dump(dump_exe, tmp_path, mesh, part, prob,
             layout=(dt, a0, a1, am, bk, kind, src.x0, src.y0, src.width, src.freq, src.amp))
    nl, mo, mc, nG, nC, n_free, nGam, max_corner = t["layout"].astype(int)
    nsub = up.nsub
    assert (nG, nC, n_free) == (up.iface.size, up.corner.size, up.free.size)
    cls = t["cls"].astype(int).reshape(nsub, nl)
    vcls = np.zeros(mesh.nn, dtype=int)
    vcls[up.free] = 1
    vcls[up.iface] = 2
    vcls[up.corner] = 3
    free_index = {int(g): k for k, g in enumerate(up.free)}
    coef = up.element_coefficients(prob)
    # local vertex of every (subdomain, row): the free vertices first in the dumped local order
    lverts = []
    for s in range(nsub):
        v = t["sub"][s]["verts"].astype(int)
        v = v[vcls[v] > 0]
        assert v.size <= nl and np.array_equal(cls[s, :v.size], vcls[v]) and np.all(cls[s, v.size:] == 0)
        assert set(v.tolist()) == set(up.subs[s]["nodes"].tolist())
        lverts.append(v)
    vert_of = lambda o: int(lverts[o // nl][o % nl])
    # pattern sizes
    npat = t["npat"].astype(int).reshape(3, nsub)
    for s in range(nsub):
        c = cls[s, :lverts[s].size]
        assert (npat[0, s], npat[1, s], npat[2, s]) == ((c == 1).sum(), (c <= 2).sum(), c.size)
    # interface / corner maps and the counting partition of unity
    owners = t["owners"].astype(int).reshape(-1, mo)[:nG]
    assert mo == max(len(up.node_subs[int(g)]) for g in up.iface)
    for g, vg in enumerate(up.iface):
        o = owners[g][owners[g] >= 0]
        assert {vert_of(x) for x in o} == {int(vg)}
        assert sorted(x // nl for x in o) == sorted(up.node_subs[int(vg)])
        assert abs(t["Dw"][g] - 1.0 / len(o)) < 1e-15
    cowners = t["cowners"].astype(int).reshape(-1, mo)[:nC]
    for c, vc in enumerate(up.corner):
        o = cowners[c][cowners[c] >= 0]
        assert {vert_of(x) for x in o} == {int(vc)} and len(o) == len(up.node_subs[int(vc)])
    gidx, cidx = t["gidx"].astype(int).reshape(nsub, nl), t["cidx"].astype(int).reshape(nsub, nl)
    gam_ln, n_gam = t["gam_ln"].astype(int).reshape(nsub, nGam), t["n_gam"].astype(int)
    loc_c, n_lc = t["loc_corner"].astype(int).reshape(nsub, mc), t["n_loc_corner"].astype(int)
    assert max_corner == n_lc.max()
    for s in range(nsub):
        v = lverts[s]
        for a in range(v.size):
            assert gidx[s, a] == (up.iface_index[int(v[a])] if cls[s, a] >= 2 else -1)
            assert cidx[s, a] == (up.corner_index[int(v[a])] if cls[s, a] == 3 else -1)
        assert gam_ln[s, :n_gam[s]].tolist() == [a for a in range(v.size) if cls[s, a] >= 2]
        assert loc_c[s, :n_lc[s]].tolist() == [a for a in range(v.size) if cls[s, a] == 3]
    # output maps
    fo, fol = t["free_owner"].astype(int), t["free_of_local"].astype(int).reshape(nsub, nl)
    for f, vf in enumerate(up.free):
        assert vert_of(fo[f]) == int(vf)
    for s in range(nsub):
        assert fol[s, :lverts[s].size].tolist() == [free_index[int(x)] for x in lverts[s]]
        assert np.all(fol[s, lverts[s].size:] == -1)
    # initial pulse (the oracle's U0, mode 0) and point load (the oracle's P1 values, split with D_s)
    usg = umesh.USGProblem(mesh, prob.replace(source=src))
    u0 = t["u0"].reshape(nsub, nl)
    U0 = usg.initial_state()[0].reshape(-1, usg.P)[:, 0] if kind == 1 else np.zeros(up.free.size)
    for s in range(nsub):
        ref = U0[[free_index[int(x)] for x in lverts[s]]]
        assert np.abs(u0[s, :lverts[s].size] - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max())
    ln_, lw = t.get("load_node", np.zeros(0)).astype(int), t.get("load_w", np.zeros(0))
    if kind == 2:
        assert ln_.size >= 3                  # the source triangle's free vertices, once per owner
        phi = umesh.p1_values(mesh, src.x0, src.y0)
        got = {}
        for o, wv in zip(ln_, lw):
            got[vert_of(o)] = got.get(vert_of(o), 0.0) + wv
            assert abs(wv * len(up.node_subs[vert_of(o)]) - src.amp * phi[vert_of(o)]) < 1e-14
        ref = {a: src.amp * v for a, v in phi.items() if a in free_index and v != 0.0}
        assert got.keys() == ref.keys()
        assert all(abs(got[a] - ref[a]) < 1e-14 for a in ref)
    else:
        assert ln_.size == 0
    # triple products
    G = pce_triple(prob)
    ptr, gi, gj, gv = t["gk_ptr"].astype(int), t["gk_i"].astype(int), t["gk_j"].astype(int), t["gk_v"]
    Gd = np.zeros_like(G)
    for k in range(G.shape[1]):
        for q in range(ptr[k], ptr[k + 1]):
            Gd[gi[q], gj[q], k] = gv[q]
    assert np.abs(Gd - G).max() < 1e-14
    # sparse rows: the oracle's subdomain mass and stiffness matrices on the free local vertices
    rp, col = t["row_ptr"].astype(int), t["col"].astype(int)
    PI = coef.shape[0]
    kv, mv = t["kval"].reshape(-1, PI), t["mval"]
    for s in range(nsub):
        v = lverts[s]
        n = v.size
        Msub, Ks = up.assemble(coef, up.subs[s]["elem_mask"])
        Mr = Msub.toarray()[np.ix_(v, v)]
        Kr = [K.toarray()[np.ix_(v, v)] for K in Ks]
        Md, Kd = np.zeros((n, n)), np.zeros((PI, n, n))
        for a in range(nl):
            row = s * nl + a
            ents = range(rp[row], rp[row + 1])
            if a >= n:
                assert len(ents) == 0
                continue
            assert col[rp[row]] == a                                  # diagonal first
            for q in ents:
                Md[a, col[q]] += mv[q]
                Kd[:, a, col[q]] += kv[q]
        assert np.abs(Md - Mr).max() <= 1e-14 * np.abs(Mr).max()
        for i in range(PI):
            assert np.abs(Kd[i] - Kr[i]).max() <= 1e-12 * np.abs(Kr[0]).max()
        # dense mean-operator inverses, pattern by pattern
        A0 = am * Mr + bk * Kr[0]
        for pat in range(3):
            inv = t[f"ainv{pat}"].reshape(nsub, nl, nl)[s]
            m = npat[pat, s]
            assert np.abs(inv[m:, :]).max(initial=0.0) == 0.0 and np.abs(inv[:, m:]).max(initial=0.0) == 0.0
            if m:
                E = inv[:m, :m] @ A0[:m, :m]
                assert np.abs(E - np.eye(m)).max() < 1e-10


def pce_triple(prob):
    from oracle import pce
    return pce.triple_products(prob.M, prob.p_in, prob.p)


@pytest.fixture(scope="module")
def rows_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("meshrows") / "mesh_rows_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", str(out), os.path.join(HERE, "helpers", "mesh_rows_check.cpp"),
                    os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_host.cpp"), "-lpthread"],
                   check=True, capture_output=True)
    return str(out)


@pytest.mark.parametrize("name,mesh,part", LAYOUT_CASES, ids=[c[0] for c in LAYOUT_CASES])
def test_mesh_kernel_rows_match_oracle(dump_exe, rows_exe, tmp_path, name, mesh, part):
    """The per-row functions the mesh kernels call (sg_mesh_rows.h), run on the host with the kernels'
    index decomposition: the SG operator apply equals cm (M (x) I) x + ck sum_i (K_i (x) G_i) x formed
    from the oracle's subdomain matrices and triple products (Sec. 4, Eq. stok), also on a CG direction
    formed on the fly (and the plain apply, to rounding, when beta = 0: the old direction, NaN here, is
    then never read), and
    the dense preconditioner solves the oracle's mean operator am M + bk K_0 on the Dirichlet and
    Neumann rows."""
    prob = w.config("small").replace(M=3, p=2, p_in=4, sigma=0.4, bx=0.4, by=0.6)
    dt, a0, a1 = 0.02, 0.3, 0.002
    am = 1.0 / (0.25 * dt * dt) + a0 * 0.5 / (0.25 * dt)
    bk = 1.0 + a1 * 0.5 / (0.25 * dt)
    layout = (dt, a0, a1, am, bk, 0, 0.5, 0.5, 0.1, 10.0, 1.0)
    t = dump(dump_exe, tmp_path, mesh, part, prob, layout=layout)
    nl = int(t["layout"][0])
    up = umesh.UPartition(mesh, part)
    nsub, P = up.nsub, prob.P
    rng = np.random.default_rng(3)
    x = rng.standard_normal((nsub, nl, P))
    wv = rng.standard_normal((nsub, nl, P))
    cm, ck = 0.7, -1.3
    (tmp_path / "x.txt").write_text(f"{cm!r} {ck!r}\n" + " ".join(f"{v:.17g}" for v in x.ravel()) + "\n" +
                                    " ".join(f"{v:.17g}" for v in wv.ravel()) + "\n")
    out = subprocess.run([rows_exe, str(tmp_path / "mesh.txt"), str(tmp_path / "layout.txt"), str(tmp_path / "x.txt")],
                         check=True, capture_output=True, text=True).stdout
    res = {ln.split()[0]: np.array([float(v) for v in ln.split()[1:]]) for ln in out.splitlines()}
    y, z0, z1, d1, d0 = (res[k].reshape(nsub, nl, P) for k in ("y", "z0", "z1", "d1", "d0"))
    coef = up.element_coefficients(prob)
    G = pce_triple(prob)
    vcls = np.zeros(mesh.nn, dtype=int)
    vcls[up.free] = 1
    vcls[up.iface] = 2
    vcls[up.corner] = 3
    for s in range(nsub):
        v = t["sub"][s]["verts"].astype(int)
        v = v[vcls[v] > 0]
        n = v.size
        Msub, Ks = up.assemble(coef, up.subs[s]["elem_mask"])
        Mr = Msub.toarray()[np.ix_(v, v)]
        Kr = [K.toarray()[np.ix_(v, v)] for K in Ks]
        X = x[s, :n]
        ref = cm * Mr @ X
        for i in range(len(Kr)):
            ref += ck * (Kr[i] @ X) @ G[i]        # [(K_i X) G_i]_{a,k} = sum_j G_ijk (K_i X_j)_a
        assert np.abs(y[s, :n] - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.all(y[s, n:] == 0.0)
        # the CG direction formed on the fly (the tensor-core loop's apply): p = x + 0.25 w, and with
        # beta 0 the old direction is never read
        Pd = X + 0.25 * wv[s, :n]
        refd = cm * Mr @ Pd
        for i in range(len(Kr)):
            refd += ck * (Kr[i] @ Pd) @ G[i]
        assert np.abs(d1[s, :n] - refd).max() <= 1e-12 * np.abs(refd).max()
        assert np.all(np.isfinite(d0[s])) and np.abs(d0[s] - y[s]).max() <= 1e-14 * np.abs(y[s]).max()
        A0 = am * Mr + bk * Kr[0]
        c = vcls[v]
        for z, m in ((z0, int((c == 1).sum())), (z1, int((c <= 2).sum()))):
            if m:
                assert np.abs(A0[:m, :m] @ z[s, :m] - X[:m]).max() <= 1e-10 * np.abs(X[:m]).max()
            assert np.all(z[s, m:] == 0.0)
