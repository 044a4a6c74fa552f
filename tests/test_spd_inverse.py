"""The host inverse of the coarse matrix F_cc (Eq. Fcc_2; csrc/sg_host.cpp, blocked Cholesky and
column solves on host threads; compiled here with g++, no GPU) against numpy: sizes below, at and
across the 64-row block boundary, condition numbers up to 1e8, an exactly symmetric result, and
rejection of matrices that are not positive definite."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def inv():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = os.path.join(ROOT, "paper_2512_23027_gb300", "_build", "spd_check")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([gxx, "-std=c++17", "-O2", "-pthread", "-o", exe, os.path.join(HERE, "helpers", "spd_check.cpp"),
                    os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_host.cpp")], check=True, capture_output=True)

    def call(A):
        n = A.shape[0]
        txt = "%d\n" % n + "\n".join(repr(float(v)) for v in A.ravel()) + "\n"
        out = subprocess.run([exe], input=txt, check=True, capture_output=True, text=True).stdout.split()
        if out[0] != "1":
            return None
        return np.array([float(v) for v in out[1:]]).reshape(n, n)
    return call


def spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n) if n > 1 else np.array([cond])
    A = (Q * ev) @ Q.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("n", [1, 2, 7, 63, 64, 65, 130, 257])
@pytest.mark.parametrize("cond", [1e2, 1e8])
def test_matches_numpy(inv, n, cond):
    A = spd(n, cond, n)
    X = inv(A)
    assert X is not None
    assert np.array_equal(X, X.T)  # mirrored, exactly symmetric
    ref = np.linalg.inv(A)
    err = np.abs(X - ref).max() / np.abs(ref).max()
    assert err <= 1e-14 * cond * max(1.0, np.sqrt(n)), err
    res = np.abs(A @ X - np.eye(n)).max()
    assert res <= 1e-13 * cond * max(1.0, np.sqrt(n)), res


def test_rejects_indefinite_and_singular(inv):
    A = spd(80, 1e3, 3)
    B = A.copy()
    B[70, 70] = -abs(B[70, 70]) - 10.0        # a negative pivot in the second block
    assert inv(B) is None
    C = np.ones((5, 5))                       # rank one: zero pivots after the first
    assert inv(C) is None


def test_coarse_like_block_matrix(inv):
    # block structure of F_cc: corners coupled through shared subdomains, P modes per corner
    rng = np.random.default_rng(11)
    nc, P = 9, 20
    n = nc * P
    A = spd(n, 1e4, 5) + np.kron(np.eye(nc), np.eye(P)) * 10.0
    X = inv(A)
    assert X is not None
    assert np.abs(A @ X - np.eye(n)).max() <= 1e-10
