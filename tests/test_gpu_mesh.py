"""GPU parity of the general-partition path (sg_setup_mesh) against the oracle's DD-PCG on the same
meshes and partitions (oracle/umesh.py; Sec. 3 corners on Delaunay meshes with 3, 5 and 6 RCB
subdomains, an island subdomain without corners, a T-junction): FP64 at PCG tolerance 1e-13 on both
sides, element by element over every free vertex and PCE mode (U within 1e-10, V 1e-9, A 1e-8
relative, the bars of the structured parity tests), with an initial pulse and with a Ricker point
source; the structured grid given as a mesh against the structured GPU solver (1e-10); mixed
precision at the workload tolerance 1e-8 (1e3 tol, iteration counts within one of the oracle's);
the one-level Neumann-Neumann and lumped preconditioners of Sec. 6.1 on a general partition (1e-10)."""
import numpy as np
import pytest

import sg_workloads as w
from oracle import dd as odd, umesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    return Solver


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def mesh_args(m, part):
    return (m.xy, m.boundary.astype(np.uint8), m.tri, np.asarray(part))


def cases():
    out = []
    m = umesh.delaunay_mesh(12, 0.3, 11)
    out += [("delaunay12_rcb3", m, umesh.rcb_partition(m, 3)), ("delaunay12_rcb5", m, umesh.rcb_partition(m, 5))]
    m = umesh.delaunay_mesh(16, 0.35, 7)
    out.append(("delaunay16_rcb6", m, umesh.rcb_partition(m, 6)))
    N = 12
    m = umesh.structured_mesh(N)
    cx, cy = (m.cen[:, 0] * N).astype(int), (m.cen[:, 1] * N).astype(int)
    out.append(("island", m, ((cx >= 4) & (cx < 8) & (cy >= 4) & (cy < 8)).astype(int)))
    out.append(("tjunction", m, np.where(cx < 6, 0, np.where(cy < 6, 1, 2))))
    return out


CASES = cases()


@pytest.mark.parametrize("src", ["pulse", "ricker"])
@pytest.mark.parametrize("name,mesh,part", CASES, ids=[c[0] for c in CASES])
def test_mesh_fp64_matches_oracle(lib, name, mesh, part, src):
    prob = w.config("small").replace(name="m", N=12, s=2, dt=0.02)
    if src == "ricker":
        prob = prob.replace(source=w.Source(2, 0.37, 0.61, 0.0, 10.0, 1.0))
    else:
        prob = prob.replace(source=w.Source(1, 0.5, 0.5, 0.15, 0.0, 1.0))
    steps = 4
    up = umesh.UPartition(mesh, part)
    usg = umesh.USGProblem(mesh, prob)
    Ur, Vr, Ar, it = odd.run_dd(usg, odd.DDSolver(prob, partition=up), steps, tol=1e-13)
    s = lib(prob, tol=1e-13, mesh=mesh_args(mesh, part))
    s.step(steps)
    U = s.field()
    state = s.get_state()
    s.close()
    n = U.size
    assert rel(U.ravel(), Ur) <= 1e-10
    assert rel(state[n:2 * n], Vr) <= 1e-9
    assert rel(state[2 * n:3 * n], Ar) <= 1e-8


def test_structured_grid_through_the_mesh_path(lib):
    """The structured grid and its s x s partition given as a mesh: the same solution as the
    structured solver (both FP64 at PCG tolerance 1e-13)."""
    prob = w.config("small")
    N, sub = prob.N, prob.s
    m = umesh.structured_mesh(N)
    H = N // sub
    ci = np.minimum((m.cen[:, 0] * N).astype(int) // H, sub - 1)
    cj = np.minimum((m.cen[:, 1] * N).astype(int) // H, sub - 1)
    part = cj * sub + ci
    a = lib(prob, tol=1e-13)
    a.step(4)
    Ua = a.field()
    a.close()
    b = lib(prob, tol=1e-13, mesh=mesh_args(m, part))
    b.step(4)
    Ub = b.field()
    b.close()
    assert rel(Ub, Ua) <= 1e-10


@pytest.mark.parametrize("name,mesh,part", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_mesh_mixed_precision(lib, name, mesh, part):
    from paper_2512_23027_gb300.binding import SG_MIXED
    prob = w.config("small").replace(name="m", N=12, s=2, dt=0.02, tol=1e-8)
    steps = 4
    up = umesh.UPartition(mesh, part)
    Ur, _, _, it = odd.run_dd(umesh.USGProblem(mesh, prob), odd.DDSolver(prob, partition=up), steps, tol=prob.tol)
    s = lib(prob, precision=SG_MIXED, mesh=mesh_args(mesh, part))
    s.step(steps)
    U = s.field()
    its, _ = s.iters()
    s.close()
    assert rel(U.ravel(), Ur) <= 1e3 * prob.tol
    assert all(abs(a - b) <= 1 for a, (b, _) in zip(its, it))


@pytest.mark.parametrize("pc", [1, 2])
def test_mesh_one_level_preconditioners(lib, pc):
    prob = w.config("small").replace(name="m", N=10, s=2, dt=0.02)
    m = umesh.delaunay_mesh(10, 0.3, 13)
    part = umesh.rcb_partition(m, 4)
    up = umesh.UPartition(m, part)
    name = {1: "nn1", 2: "lumped"}[pc]
    Ur, _, _, it = odd.run_dd(umesh.USGProblem(m, prob), odd.DDSolver(prob, partition=up, precond=name), 2,
                              tol=1e-13)
    s = lib(prob, tol=1e-13, precond=pc, mesh=mesh_args(m, part))
    s.step(2)
    U = s.field()
    s.close()
    assert rel(U.ravel(), Ur) <= 1e-10
