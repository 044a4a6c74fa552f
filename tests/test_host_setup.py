"""The library's host set-up (csrc/sg_host.cpp, compiled here with g++ into a small dump program; no
GPU) against the oracle, table by table:
- KL eigenvalues (Sec. 4, Eq. KLE);
- the output multi-indices;
- the Hermite triple products G_ijk grouped by output mode (Sec. 4), with exactly the oracle's
  nonzeros;
- the node classes and interface numbering of the partition (Sec. 3);
- the counting weights D_s;
- the stiffness edge weights of every subdomain.  In the graph-Laplacian form of P1 on right
  triangles, the weight of edge (a, b) in subdomain s is -K_i^(s)[a, b], where K_i^(s) is the
  stiffness the oracle assembles over that subdomain's elements (Sec. 4, Eq. stok);
- the source terms: the point load's P1 weights, split over the subdomains that hold the node
  (counting weights, Sec. 3), and the interpolated initial pulse (Sec. 6.2)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import sg_workloads as w
from oracle import dd, fem, kl, pce

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (N, s, M, p, p_in): a 2 x 2 and a 3 x 3 partition, P = 20 and 15, and an input order 2p
CASES = [(24, 3, 2, 2, 2), (32, 2, 2, 2, 2), (24, 2, 3, 3, 3), (16, 4, 4, 2, 2), (12, 2, 2, 2, 4)]
CLS = {"i": 1, "r": 2, "c": 3}


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("host") / "host_dump"
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", str(out), os.path.join(HERE, "helpers", "host_dump.cpp"),
                    os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_host.cpp")],
                   check=True, capture_output=True)
    return str(out)


def host_tables(exe, prob):
    src = prob.source
    args = [prob.N, prob.s, prob.M, prob.sigma, prob.bx, prob.by, prob.g0, prob.p, prob.p_in, prob.dt,
            src.kind, src.x0, src.y0, src.width, src.freq, src.amp]
    txt = subprocess.run([exe] + [repr(a) for a in args], check=True, capture_output=True, text=True).stdout
    t = {}
    for line in txt.splitlines():
        name, *vals = line.split()
        t[name] = np.array([float(v) for v in vals])
    L, nl, nsub, P, PI, nG, nC, n_free = map(int, t["sizes"])
    t.update(L=L, nl=nl, nsub=nsub, P=P, PI=PI, nG=nG, nC=nC, n_free=n_free)
    return t


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "N%d_s%d_M%d_p%d_pin%d" % c)
def case(request, dump_exe):
    N, s, M, p, p_in = request.param
    prob = w.config("small").replace(N=N, s=s, M=M, p=p, p_in=p_in, sigma=0.3, bx=0.4, by=0.6, dt=w.cfl_dt(N))
    return prob, host_tables(dump_exe, prob)


def test_kl_eigenvalues(case):
    prob, t = case
    ref = np.array([lam for lam, _, _ in kl.kl_modes(prob.M, prob.bx, prob.by)])
    assert np.allclose(t["kl_lambda"], ref, rtol=1e-12, atol=0)


def test_multi_indices(case):
    prob, t = case
    ref = np.array(pce.multi_indices(prob.M, prob.p))
    assert t["P"] == len(ref) and np.array_equal(t["alpha_out"].reshape(len(ref), prob.M), ref)


def test_triple_products(case):
    prob, t = case
    ref = pce.triple_products(prob.M, prob.p_in, prob.p)           # [i, j, k]
    PI, P = t["PI"], t["P"]
    assert ref.shape == (PI, P, P)
    G = np.zeros_like(ref)
    ptr = t["gk_ptr"].astype(int)
    gi, gj, gv = t["gk_i"].astype(int), t["gk_j"].astype(int), t["gk_v"]
    for k in range(P):
        for q in range(ptr[k], ptr[k + 1]):
            assert G[gi[q], gj[q], k] == 0.0    # each triple once
            G[gi[q], gj[q], k] = gv[q]
    assert np.array_equal(G != 0.0, ref != 0.0)
    assert np.allclose(G, ref, rtol=1e-14, atol=1e-15)


def test_partition_classes_and_interface(case):
    prob, t = case
    part = dd.Partition(prob.N, prob.s)
    N, s, H, L, nl = prob.N, prob.s, prob.N // prob.s, t["L"], t["nl"]
    assert (t["nG"], t["nC"], t["n_free"]) == (part.iface.size, part.corner.size, part.free.size)
    cls, gidx = t["cls"].astype(int), t["gidx"].astype(int)
    for sub_id, sub in enumerate(part.subs):
        sy, sx = divmod(sub_id, s)
        ocls = dict(zip(sub["nodes"].tolist(), sub["cls"].tolist()))
        for lj in range(L):
            for li in range(L):
                g = fem.node_id(sx * H + li, sy * H + lj, N)
                o = sub_id * nl + lj * L + li
                assert cls[o] == (CLS[ocls[g]] if g in ocls else 0)
                assert gidx[o] == part.iface_index.get(g, -1)
    assert np.allclose(t["Dw"], 1.0 / part.mult, rtol=0, atol=1e-15)


def test_edge_weights_equal_minus_the_subdomain_stiffness(case):
    prob, t = case
    part = dd.Partition(prob.N, prob.s)
    N, s, H, L, nl, PI = prob.N, prob.s, prob.N // prob.s, t["L"], t["nl"], t["PI"]
    coef = fem.element_coefficients(prob)
    kapE = t["kapE"].reshape(t["nsub"], nl, PI)
    kapN = t["kapN"].reshape(t["nsub"], nl, PI)
    li, lj = np.meshgrid(np.arange(L), np.arange(L))
    li, lj = li.ravel(), lj.ravel()
    for sub_id, sub in enumerate(part.subs):
        sy, sx = divmod(sub_id, s)
        _, Ks = fem.assemble(N, coef, elem_mask=sub["elem_mask"])
        I, J = sx * H + li, sy * H + lj
        a = fem.node_id(I, J, N)
        e_ok, n_ok = li < H, lj < H
        for i in range(PI):
            K = Ks[i].tocsr()
            refE = np.zeros(nl)
            refN = np.zeros(nl)
            refE[e_ok] = -np.asarray(K[a[e_ok], fem.node_id(I[e_ok] + 1, J[e_ok], N)]).ravel()
            refN[n_ok] = -np.asarray(K[a[n_ok], fem.node_id(I[n_ok], J[n_ok] + 1, N)]).ravel()
            scale = max(np.abs(refE).max(), np.abs(refN).max(), 1e-300)
            assert np.allclose(kapE[sub_id, :, i], refE, rtol=0, atol=1e-13 * scale)
            assert np.allclose(kapN[sub_id, :, i], refN, rtol=0, atol=1e-13 * scale)


def _global_of_local(prob, nl, L, o):
    sub_id, ln = divmod(int(o), nl)
    sy, sx = divmod(sub_id, prob.s)
    lj, li = divmod(ln, L)
    H = prob.N // prob.s
    return fem.node_id(sx * H + li, sy * H + lj, prob.N)


# Ricker point sources: inside a subdomain, on an interface line (node held by 2 subdomains) and on a
# cross point (4 subdomains); 24^2 grid, 3 x 3 subdomains (interface lines at 8 and 16 cells)
@pytest.mark.parametrize("x0,y0", [(0.3, 0.5), (1.0 / 3.0, 0.5 + 0.01), (1.0 / 3.0, 2.0 / 3.0)])
def test_point_load_weights(dump_exe, x0, y0):
    base = w.config("small")
    prob = base.replace(source=base.source.__class__(2, x0, y0, 0.0, 10.0, 1.7))
    t = host_tables(dump_exe, prob)
    part = dd.Partition(prob.N, prob.s)
    held = {}
    for sub in part.subs:
        for g in sub["nodes"].tolist():
            held[g] = held.get(g, 0) + 1
    ref = {g: prob.source.amp * v for g, v in fem.p1_values(prob.N, x0, y0).items() if g in part.free_index}
    got = {}
    for o, wgt in zip(t["load_node"], t["load_w"]):
        g = _global_of_local(prob, t["nl"], t["L"], o)
        assert np.isclose(wgt, ref[g] / held[g], rtol=1e-15, atol=0)
        got[g] = got.get(g, 0.0) + wgt
    assert set(got) == set(ref)
    assert all(np.isclose(got[g], ref[g], rtol=1e-14, atol=0) for g in ref)
    assert max(held[g] for g in ref) > 1 or (x0, y0) == (0.3, 0.5)


def test_initial_pulse(dump_exe):
    base = w.config("small")
    prob = base.replace(source=base.source.__class__(1, 0.45, 0.55, 0.1, 0.0, 1.3))
    t = host_tables(dump_exe, prob)
    ref = fem.initial_displacement(prob.N, prob.source)
    part = dd.Partition(prob.N, prob.s)
    u0 = t["u0_local"]
    for o in range(u0.size):
        g = _global_of_local(prob, t["nl"], t["L"], o)
        assert np.isclose(u0[o], ref[g] if g in part.free_index else 0.0, rtol=1e-14, atol=1e-300)


def _centroids(N):
    _, cen = fem.elements(N)
    return cen


def _write_kl(path, lam, modes):
    with open(path, "w") as f:
        f.write(" ".join(repr(float(v)) for v in lam) + "\n")
        f.write(" ".join(repr(float(v)) for v in np.ravel(modes)) + "\n")


def host_tables_kl(exe, prob, lam, modes, path):
    _write_kl(path, lam, modes)
    src = prob.source
    args = [prob.N, prob.s, prob.M, prob.sigma, prob.bx, prob.by, prob.g0, prob.p, prob.p_in, prob.dt,
            src.kind, src.x0, src.y0, src.width, src.freq, src.amp]
    txt = subprocess.run([exe] + [repr(a) for a in args] + [str(path)], check=True, capture_output=True,
                         text=True).stdout
    return {line.split()[0]: np.array([float(v) for v in line.split()[1:]]) for line in txt.splitlines()}


def test_caller_kl_modes_analytic_equal_built_in(dump_exe, tmp_path):
    """The analytic eigenpairs passed in as caller modes (the oracle's phi_n at the element centroids
    and its lambda_n) give the tables of the built-in analytic KL."""
    prob = w.config("small")
    cen = _centroids(prob.N)
    lam, phi = [], []
    for lm, (ix, wx, px), (iy, wy, py) in kl.kl_modes(prob.M, prob.bx, prob.by):
        lam.append(lm)
        phi.append(kl.phi1d(cen[:, 0], wx, px) * kl.phi1d(cen[:, 1], wy, py))
    a = host_tables(dump_exe, prob)
    b = host_tables_kl(dump_exe, prob, lam, np.array(phi), tmp_path / "kl.txt")
    assert np.allclose(b["kl_lambda"], a["kl_lambda"], rtol=1e-15, atol=0)
    for t in ("kapE", "kapN"):
        assert np.allclose(b[t], a[t], rtol=1e-12, atol=1e-15 * np.abs(a[t]).max())


def test_caller_kl_modes_reach_the_edge_weights(dump_exe, tmp_path):
    """Caller modes that are neither separable nor symmetric (the analytic modes times
    1 + 0.3 sin(7x + 3y), an arbitrary positive lambda): every subdomain's edge weights equal minus
    the oracle's stiffness entries assembled from the PCE of exp(g), g_n = sigma sqrt(lambda_n) phi_n
    at the same centroids (a wrong element order, a T1 / T2 swap or a scaling slip fails this)."""
    prob = w.config("small").replace(M=2, p=2, p_in=2)
    N, s, H = prob.N, prob.s, prob.N // prob.s
    cen = _centroids(N)
    bump = 1.0 + 0.3 * np.sin(7 * cen[:, 0] + 3 * cen[:, 1])
    lam = [0.37, 0.11]
    phi = []
    for lm, (ix, wx, px), (iy, wy, py) in kl.kl_modes(prob.M, prob.bx, prob.by):
        phi.append(kl.phi1d(cen[:, 0], wx, px) * kl.phi1d(cen[:, 1], wy, py) * bump)
    phi = np.array(phi)
    t = host_tables_kl(dump_exe, prob, lam, phi, tmp_path / "kl.txt")
    from oracle import field
    gn = prob.sigma * np.sqrt(np.array(lam))[:, None] * phi
    coef = field.lognormal_pce(gn, prob.g0, prob.p_in)
    part = dd.Partition(N, s)
    L = H + 1
    PI = coef.shape[0]
    kapE = t["kapE"].reshape(s * s, L * L, PI)
    kapN = t["kapN"].reshape(s * s, L * L, PI)
    worst = 0.0
    for si, sub in enumerate(part.subs):
        _, Ks = fem.assemble(N, coef, sub["elem_mask"])
        sx, sy = si % s, si // s
        for lj in range(L):
            for li in range(L):
                I, J = sx * H + li, sy * H + lj
                a = fem.node_id(I, J, N)
                for i in range(PI):
                    if li < H:
                        ref = -Ks[i][a, fem.node_id(I + 1, J, N)]
                        worst = max(worst, abs(kapE[si, lj * L + li, i] - ref))
                    if lj < H:
                        ref = -Ks[i][a, fem.node_id(I, J + 1, N)]
                        worst = max(worst, abs(kapN[si, lj * L + li, i] - ref))
    assert worst < 1e-13, worst
