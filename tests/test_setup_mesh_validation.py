"""sg_setup_mesh rejects invalid and unsupported meshes, partitions and parameters before its first
CUDA call (no device needed): each failure returns its status code with a message in
sg_last_error(NULL) and leaves the output handle NULL.  On a machine without a GPU, a valid mesh
passes every host step (mesh tables, corner detection, sparse rows, index checks, the dense
mean-operator inverses) and stops at the first CUDA call with SG_ECUDA."""
import ctypes as C

import numpy as np
import pytest

import sg_workloads as w
from oracle import umesh

SG_EINVAL, SG_ECUDA, SG_ENOTSUP = -1, -3, -7


@pytest.fixture(scope="module")
def B():
    from paper_2512_23027_gb300 import build as b
    b.build()
    from paper_2512_23027_gb300 import binding
    binding.load_library()
    return binding


def base_mesh():
    m = umesh.delaunay_mesh(6, 0.3, 5)
    return m.xy.copy(), m.boundary.astype(np.uint8), m.tri.astype(np.int32).copy(), umesh.rcb_partition(m, 3).astype(np.int32)


def setup_rc(B, xy, dirichlet, tri, part, precision=0, warm=0, src=None, modes=None, lambdas=None, null_mesh=False,
             prob=None, precond=0):
    lib = B.load_library()
    prob = prob or w.config("tiny")
    s = src or prob.source
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    mesh = B.Mesh(xy.shape[0], xy.ctypes.data, dirichlet.ctypes.data, tri.shape[0], tri.ctypes.data,
                  part.ctypes.data)
    kl = B.KL(prob.M, prob.sigma, prob.bx, prob.by, prob.g0, None if modes is None else modes.ctypes.data,
              None if lambdas is None else lambdas.ctypes.data)
    pce = B.PCE(prob.p, prob.p_in)
    prm = B.Params(prob.dt, prob.tol, prob.alpha0, prob.alpha1, prob.max_iter, precision, warm, 0.0, 0, 0, 0, 0.0,
                   precond)
    srcs = B.Source(s.kind, s.x0, s.y0, s.width, s.freq, s.amp)
    h = C.c_void_p(12345)
    rc = lib.sg_setup_mesh(None if null_mesh else C.byref(mesh), C.byref(kl), C.byref(pce), C.byref(prm),
                           C.byref(srcs), None, C.byref(h))
    return rc, h.value, lib.sg_last_error(None).decode()


def bad(kind):
    xy, d, tri, part = base_mesh()
    kw = {}
    if kind == "vertex id":
        tri[3, 1] = xy.shape[0]
    elif kind == "unused subdomain id":
        part = np.where(part == 1, 2, part)
    elif kind == "single subdomain":
        part = np.zeros_like(part)
    elif kind == "degenerate triangle":
        xy[tri[0, 2]] = 0.5 * (xy[tri[0, 0]] + xy[tri[0, 1]])
    elif kind == "edge in three triangles":
        a, b = tri[0, 0], tri[0, 1]
        xy = np.vstack([xy, [[0.5, 0.5]]])
        d = np.append(d, 0)
        tri = np.vstack([tri, [[a, b, xy.shape[0] - 1]]])
        part = np.append(part, 0)
    elif kind == "source outside the mesh":
        xy = 0.5 * xy                       # the mesh covers [0, 1/2]^2 only
        kw["src"] = w.Source(2, 0.8, 0.8, 0.0, 10.0, 1.0)
    elif kind == "source kind":
        kw["src"] = w.Source(5, 0.5, 0.5, 0.05, 10.0, 1.0)
    elif kind == "precision":
        kw["precision"] = 7
    elif kind == "bf16 with P > 32":
        kw["precision"] = 3
        kw["prob"] = w.config("tiny").replace(M=4, p=3, p_in=3)    # P = 35
    elif kind == "warm-start mode":
        kw["warm"] = 9
    elif kind == "modes without lambdas":
        kw["modes"] = np.zeros((w.config("tiny").M, tri.shape[0]))
    elif kind == "too few vertices":
        xy, d = xy[:2], d[:2]
    elif kind == "subdomain too large":
        from sg_workloads import meshes
        xy, tri, bnd = meshes.delaunay_square(100, 0.3, 5)     # 10201 vertices in 2 subdomains
        d = bnd.astype(np.uint8)
        part = meshes.rcb_partition(xy, tri, 2)
    return (xy, d, tri, part), kw


CASES = [
    ("vertex id", SG_EINVAL, "out of range"),
    ("unused subdomain id", SG_EINVAL, "subdomain ids"),
    ("single subdomain", SG_ENOTSUP, "two subdomains"),
    ("degenerate triangle", SG_EINVAL, "degenerate"),
    ("edge in three triangles", SG_EINVAL, "more than two"),
    ("source outside the mesh", SG_EINVAL, "no triangle"),
    ("source kind", SG_EINVAL, "source"),
    ("precision", SG_EINVAL, "precision"),
    ("bf16 with P > 32", SG_ENOTSUP, "SG_BF16"),
    ("warm-start mode", SG_EINVAL, "warm"),
    ("modes without lambdas", SG_EINVAL, "lambdas"),
    ("too few vertices", SG_EINVAL, "mesh"),
    ("subdomain too large", SG_ENOTSUP, "at most 4096"),
]


@pytest.mark.parametrize("kind,code,msg", CASES, ids=[c[0] for c in CASES])
def test_mesh_setup_rejects(B, kind, code, msg):
    args, kw = bad(kind)
    rc, h, err = setup_rc(B, *args, **kw)
    assert rc == code and h is None and msg in err, (rc, err)


def test_null_mesh(B):
    rc, h, err = setup_rc(B, *base_mesh(), null_mesh=True)
    assert rc == SG_EINVAL and h is None and "null" in err


def test_valid_mesh_passes_the_host_steps(B):
    """Without a GPU the first CUDA call fails: every host step before it accepted the mesh (an RCB
    partition of a Delaunay mesh into three subdomains, which meet at a corner; pulse and Ricker
    sources; FP64, mixed precision and SG_BF16 (its tensor-core image is built after the first CUDA
    call); the two-level and the one-level preconditioner, whose third pattern adds one more
    mean-operator inverse)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible: this checks the host steps on a machine without one")
    for src in (w.Source(1, 0.5, 0.5, 0.1, 0.0, 1.0), w.Source(2, 0.37, 0.61, 0.0, 10.0, 1.0)):
        for precision, precond in ((0, 0), (1, 0), (0, 1), (3, 0)):
            rc, h, err = setup_rc(B, *base_mesh(), src=src, precision=precision, precond=precond)
            assert rc == SG_ECUDA and h is None, (rc, err)


@pytest.mark.parametrize("name,nv,nsub", [("umesh_small", 625, 6), ("umesh13k", 13689, 32), ("umesh37k", 37249, 64),
                                          ("umesh37k_720", 37249, 720), ("umesh_e1", 1600, 4)])
def test_mesh_workloads(B, name, nv, nsub):
    """The mesh workloads: seeded (the same mesh twice), the vertex counts of the paper-sized meshes,
    balanced RCB partitions (triangle counts within one), and every host step of sg_setup_mesh accepts
    them (on a machine without a GPU the set-up stops at the first CUDA call)."""
    c = w.mesh_config(name)
    xy, d, tri, part = c.build()
    xy2, _, tri2, part2 = c.build()
    assert np.array_equal(xy, xy2) and np.array_equal(tri, tri2) and np.array_equal(part, part2)
    assert xy.shape[0] == nv and int(part.max()) + 1 == nsub
    cnt = np.bincount(part, minlength=nsub)
    assert cnt.max() - cnt.min() <= 1
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        return
    rc, h, err = setup_rc(B, xy, d, tri, part, prob=c.prob, precision=1)
    assert rc == SG_ECUDA and h is None, (rc, err)


def test_mesh_golden_matches_the_generator():
    """The stored oracle samples of the 37k-vertex mesh workload (tests/golden/mesh_oracle_samples.json)
    were taken on the mesh and partition that sg_workloads builds here (sha256 of the sorted triangles
    and of the partition), with the sample layout the GPU test reads."""
    import importlib.util
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "golden", "mesh_oracle_samples.json")
    if not os.path.exists(path):
        pytest.skip("mesh_oracle_samples.json not generated")
    spec = importlib.util.spec_from_file_location("mk", os.path.join(here, "golden", "make_mesh_oracle_samples.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    rec = json.load(open(path))["umesh37k"]
    xy, d, tri, part = w.mesh_config("umesh37k").build()
    assert mk.mesh_hash(tri, part) == (rec["mesh_sha"], rec["part_sha"])
    assert rec["vertices"] == xy.shape[0] and rec["triangles"] == tri.shape[0]
    n = len(rec["node"])
    assert n == len(rec["mode"]) == len(rec["tight"]["values"]) == len(rec["workload"]["values"])
    assert max(rec["node"]) < rec["n_free"] and max(rec["mode"]) < w.mesh_config("umesh37k").prob.P
    assert rec["tight"]["tol"] == 1e-13 and len(rec["tight"]["iters"]) == rec["steps"]


def test_mesh_plan_query_matches_the_oracle_partition(B):
    """sg_mesh_plan_query (host-only) reports the partition's sizes as the oracle's UPartition counts them
    (free, interface and corner vertices, the largest subdomain, multiplicities, local corners and
    interface vertices), the sparse-row entries (diagonal plus the free neighbours along triangle edges,
    per subdomain), the coarse order n_corner * P, and byte counts that follow from them."""
    from oracle import umesh
    c = w.mesh_config("umesh_small")
    xy, d, tri, part = c.build()
    up = umesh.UPartition(umesh.Mesh(xy, tri, d), part)
    p = c.prob
    plan = B.mesh_plan_query(p, (xy, d, tri, part), precision=0)
    assert (plan["nsub"], plan["n_free"], plan["n_gamma"], plan["n_corner"]) == \
        (up.nsub, up.free.size, up.iface.size, up.corner.size)
    nl = max(s["nodes"].size for s in up.subs)
    assert plan["n_sub_nodes"] == nl and plan["P"] == p.P
    assert plan["max_owners"] == max(len(up.node_subs[int(g)]) for g in up.iface)
    assert plan["max_corners"] == max(int((s["cls"] == "c").sum()) for s in up.subs)
    assert plan["max_gamma"] == max(s["gamma"].size for s in up.subs)
    free = set(up.free.tolist())
    entries = 0
    for s in range(up.nsub):
        pairs = set()
        for t in tri[part == s]:
            for a in t:
                for b in t:
                    if int(a) in free and int(b) in free:
                        pairs.add((int(a), int(b)))
        entries += len(pairs)
    assert plan["row_entries"] == entries
    assert plan["coarse_dim"] == up.corner.size * p.P
    assert plan["bytes_coarse_matrix"] == (up.corner.size * p.P) ** 2 * 8
    assert plan["bytes_inverses"] == 2 * up.nsub * nl * nl * 8 and plan["mma"] == 0 and plan["fits"] == 1
    mixed = B.mesh_plan_query(p, (xy, d, tri, part), precision=1)
    assert mixed["bytes_inverses"] == 2 * up.nsub * nl * nl * 4
    bf16 = B.mesh_plan_query(p, (xy, d, tri, part), precision=3)
    kp = (nl + 127) // 128 * 128
    assert bf16["mma"] == 1 and bf16["bytes_inverses"] == mixed["bytes_inverses"] + 2 * up.nsub * kp * kp * 2
    nn1 = B.mesh_plan_query(p, (xy, d, tri, part), precision=0, precond=1)
    assert nn1["bytes_inverses"] == 3 * up.nsub * nl * nl * 8 and nn1["bytes_coarse_matrix"] == 0


def test_mesh_plan_query_of_the_paper_partition(B):
    """The 37k-vertex mesh on the paper's 720 subdomains: 1284 corners, a coarse matrix of order 25680
    (5.3 GB dense) at P = 20; on 64 subdomains 49 corners."""
    for name, corners in (("umesh37k_720", 1284), ("umesh37k", 49)):
        c = w.mesh_config(name)
        plan = B.mesh_plan_query(c.prob, c.build())
        assert plan["n_corner"] == corners and plan["coarse_dim"] == corners * 20
        assert plan["bytes_coarse_matrix"] == (corners * 20) ** 2 * 8 and plan["fits"] == 1
    # two subdomains of a 10201-vertex mesh exceed the dense inverse's 4096 free vertices
    from sg_workloads import meshes
    xy, tri, bnd = meshes.delaunay_square(100, 0.3, 5)
    plan = B.mesh_plan_query(w.config("tiny"), (xy, bnd.astype(np.uint8), tri, meshes.rcb_partition(xy, tri, 2)))
    assert plan["n_sub_nodes"] > 4096 and plan["fits"] == 0


@pytest.mark.parametrize("n,seed,nparts", [(12, 11, 3), (12, 11, 5), (24, 11, 6), (39, 61, 17), (192, 37, 64),
                                           (192, 37, 720)])
def test_native_rcb_partition_equals_the_generator(B, n, seed, nparts):
    """sg_partition_rcb (C++, host) gives the same partition as the workloads' RCB (sg_workloads.meshes),
    element for element, with balanced triangle counts."""
    from sg_workloads import meshes
    xy, tri, _ = meshes.delaunay_square(n, 0.3, seed)
    ref = meshes.rcb_partition(xy, tri, nparts)
    got = B.partition_rcb(xy, tri, nparts)
    assert np.array_equal(got, ref)
    cnt = np.bincount(got, minlength=nparts)
    assert cnt.size == nparts and cnt.min() >= 1 and cnt.max() - cnt.min() <= 1


def test_native_rcb_partition_rejects(B):
    from sg_workloads import meshes
    xy, tri, _ = meshes.delaunay_square(6, 0.3, 5)
    for nparts in (0, tri.shape[0] + 1):
        with pytest.raises(B.SGError):
            B.partition_rcb(xy, tri, nparts)
    bad = tri.copy()
    bad[0, 0] = xy.shape[0]
    with pytest.raises(B.SGError):
        B.partition_rcb(xy, bad, 3)


def test_binding_marshals_the_mesh(B):
    """Solver(prob, mesh=...) passes the mesh arrays through sg_setup_mesh: on a machine without a GPU the
    host steps accept them and the set-up stops at the first CUDA call (SGError with SG_ECUDA)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible: this checks the host steps on a machine without one")
    from paper_2512_23027_gb300 import Solver
    c = w.mesh_config("umesh_small")
    with pytest.raises(B.SGError) as e:
        Solver(c.prob, precision=1, mesh=c.build())
    assert e.value.code == SG_ECUDA
