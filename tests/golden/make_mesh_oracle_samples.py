"""Writes tests/golden/mesh_oracle_samples.json: seeded samples of the CPU oracle's DD-PCG results on a
mesh workload too large for the oracle to finish inside a GPU test run (umesh37k: 37249 vertices, 64
RCB subdomains, M = 3, order 3, P = 20; the oracle needs about four minutes of set-up and half a
minute per step on 8 x86 cores).

Only the oracle (oracle/) and the workload inputs (sg_workloads) are used.  The oracle advances
`steps` Newmark steps twice, at PCG tolerance 1e-13 (the FP64 parity setting) and at the workload
tolerance, and records per run: the outer iteration counts per step, the l2 norm of every PCE mode
of U over the free vertices, and the values of U at a sample of (free vertex, mode) entries: half
drawn uniformly (numpy default_rng, seed 20251227), half the entries of largest magnitude of the
tight run's field.  It also records a sha256 of the mesh (sorted triangles) and of the partition:
the Delaunay triangulation comes from scipy, so a test on another platform first checks that it
rebuilt the same mesh.

Run: python tests/golden/make_mesh_oracle_samples.py
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sg_workloads as w  # noqa: E402
from oracle import dd, umesh  # noqa: E402

NSAMPLE = 2048
STEPS = 3


def mesh_hash(tri, part):
    """sha256 prefixes of the triangle set (vertex ids sorted per triangle, triangles sorted) and of the
    partition in that order."""
    t = np.sort(np.asarray(tri, dtype=np.int64), axis=1)
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    ht = hashlib.sha256(np.ascontiguousarray(t[order]).tobytes()).hexdigest()[:16]
    hp = hashlib.sha256(np.ascontiguousarray(np.asarray(part, dtype=np.int64)[order]).tobytes()).hexdigest()[:16]
    return ht, hp


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mesh_oracle_samples.json")
    out = {}
    for name in ("umesh37k",):
        t0 = time.time()
        c = w.mesh_config(name)
        xy, boundary, tri, part = c.build()
        prob = c.prob
        m = umesh.Mesh(xy, tri, boundary)
        up = umesh.UPartition(m, part)
        usg = umesh.USGProblem(m, prob)
        solver = dd.DDSolver(prob, partition=up)
        runs = {}
        for label, tol in (("tight", 1e-13), ("workload", prob.tol)):
            U, _, _, it = dd.run_dd(usg, solver, STEPS, tol=tol)
            runs[label] = (U.reshape(-1, prob.P), [int(i) for i, _ in it])
        nf = up.free.size
        rng = np.random.default_rng(20251227)
        flat = np.argsort(-np.abs(runs["tight"][0]).ravel(), kind="stable")[: NSAMPLE // 2]
        node = np.concatenate([rng.integers(0, nf, NSAMPLE // 2), flat // prob.P])
        mode = np.concatenate([rng.integers(0, prob.P, NSAMPLE // 2), flat % prob.P])
        ht, hp = mesh_hash(tri, part)
        rec = {"workload": name, "mesh_sha": ht, "part_sha": hp, "vertices": int(xy.shape[0]),
               "triangles": int(tri.shape[0]), "n_free": int(nf), "steps": STEPS, "n_uniform": NSAMPLE // 2,
               "node": node.tolist(), "mode": mode.tolist()}
        for label, tol in (("tight", 1e-13), ("workload", prob.tol)):
            U, its = runs[label]
            rec[label] = {"tol": tol, "iters": its, "mode_norm": np.linalg.norm(U, axis=0).tolist(),
                          "norm": float(np.linalg.norm(U)), "values": U[node, mode].tolist()}
        out[name] = rec
        json.dump(out, open(path, "w"), separators=(",", ":"))
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
