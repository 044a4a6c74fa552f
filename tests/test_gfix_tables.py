"""The compile-time triple-product tables of the FP32 operator apply (sg_gfix.cuh) against the
oracle: for every compiled (M, p, p_in), the nonzero triples (i, j, k) of the normalised Hermite
triple products, in the order output mode k, then input mode i, then mode j, are exactly those of
oracle.pce.triple_products (Sec. 4, G_ijk), and the PCE sizes match C(M + p, p).  The tables are
printed by a host-only program compiled with nvcc (no GPU needed)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import pce

HERE = os.path.dirname(os.path.abspath(__file__))


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    exe = nvcc()
    if exe is None:
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("gfix") / "gfix_dump"
    subprocess.run([exe, "-std=c++17", "-O1", "-o", str(out), os.path.join(HERE, "helpers", "gfix_dump.cu")],
                   check=True, capture_output=True)
    lines = subprocess.run([str(out)], check=True, capture_output=True, text=True).stdout.split("\n")
    res, pos = [], 0
    while pos < len(lines) and lines[pos].strip():
        M, p, pin, P, PI, nnz = map(int, lines[pos].split())
        ent = [tuple(map(int, lines[pos + 1 + e].split())) for e in range(nnz)]
        res.append((M, p, pin, P, PI, ent))
        pos += 1 + nnz
    return res


def test_compiled_sizes_cover_the_workloads(tables):
    have = {(M, p, pin) for M, p, pin, *_ in tables}
    for mp in [(2, 2), (2, 3), (3, 2), (3, 3), (4, 2), (4, 3), (5, 2)]:
        assert (mp[0], mp[1], mp[1]) in have


def test_tables_match_oracle(tables):
    for M, p, pin, P, PI, ent in tables:
        assert P == math.comb(M + p, p) and PI == math.comb(M + pin, pin)
        G = pce.triple_products(M, pin, p)                      # [i][j][k]
        ref = [(i, j, k) for k in range(P) for i in range(PI) for j in range(P) if abs(G[i, j, k]) > 0.0]
        assert ent == ref, (M, p, pin)
        # every listed entry is nonzero and none is missing
        assert all(abs(G[i, j, k]) > 0.0 for i, j, k in ent)
        assert len(ent) == int(np.count_nonzero(np.abs(G) > 0.0))
