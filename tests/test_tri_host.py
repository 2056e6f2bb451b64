"""CPU checks of the device helpers behind the Rayleigh-Ritz eigensolvers
(csrc/tri_common.cuh, built for the host by nvcc): the Sturm count by the
signs of the leading principal minors and by the LDL^T pivots, against the
eigenvalues numpy computes, including the cases random matrices never reach
(a minor that is exactly zero, decoupled blocks, chains long enough to need
rescaling); inverse iteration (one factorization, three solves) against
numpy's eigenvectors, with and without row interchanges.  Also the device
Philox4x32-10 against the published known-answer vectors (the oracle's own
Philox is pinned to the same vectors in test_oracle_eig.py)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "tri_harness.cu")
OUT = os.path.join(HERE, "host", "_build", "libtri_harness.so")


@pytest.fixture(scope="module")
def lib():
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", SRC, "-o", OUT])
    L = C.CDLL(OUT)
    dp = C.POINTER(C.c_double)
    L.h_count_minors.argtypes = [dp, dp, C.c_int, C.c_double]
    L.h_count_ratio.argtypes = [dp, dp, C.c_int, C.c_double, C.c_double]
    L.h_inv_iter.argtypes = [dp, dp, C.c_int, C.c_double, dp, dp, C.c_int]
    L.h_inv_iter.restype = None
    up = C.POINTER(C.c_uint)
    L.h_philox.argtypes = [up, C.c_uint, C.c_uint, up]
    L.h_philox.restype = None
    return L


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def tridiag(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def counts(lib, d, e, x):
    d = np.ascontiguousarray(d, dtype=np.float64)
    e2 = np.ascontiguousarray(np.append(np.asarray(e, dtype=np.float64) ** 2, 0.0))
    return (lib.h_count_minors(_p(d), _p(e2), len(d), float(x)),
            lib.h_count_ratio(_p(d), _p(e2), len(d), float(x), 2.2250738585072014e-308))


def random_unit_tridiag(rng, p):
    d, e = rng.uniform(-1, 1, p), rng.uniform(-1, 1, p - 1)
    lam = np.linalg.eigvalsh(tridiag(d, e))
    s = np.abs(lam).max()
    return d / s, e / s


@pytest.mark.parametrize("p", [1, 2, 7, 64, 300])
def test_sturm_counts_equal_the_eigenvalue_count(lib, p):
    rng = np.random.default_rng(p)
    for _ in range(3):
        d, e = random_unit_tridiag(rng, p) if p > 1 else (rng.uniform(-1, 1, 1), np.zeros(0))
        lam = np.sort(np.linalg.eigvalsh(tridiag(d, e)))
        gaps = np.diff(lam)
        xs = list(rng.uniform(-1.01, 1.01, 40)) + [-1.01, 1.01]
        if p > 1:  # midpoints between neighbouring eigenvalues
            xs += list(0.5 * (lam[:-1] + lam[1:])[gaps > 1e-9][:40])
        for x in xs:
            if np.min(np.abs(lam - x)) < 1e-10:
                continue  # within rounding of an eigenvalue: either count is right
            want = int(np.sum(lam < x))
            assert counts(lib, d, e, x) == (want, want), (p, x)


def test_zero_minor_takes_the_sign_opposite_to_its_predecessor(lib):
    # x equal to an eigenvalue of a leading block makes that minor exactly 0;
    # the count must still be the number of eigenvalues below x
    d = np.array([0.25, -0.5, 0.75, 0.1])
    e = np.array([0.0, 0.3, 0.2])  # first row decoupled: f_1 = d_0 - x = 0 at x = 0.25
    lam = np.sort(np.linalg.eigvalsh(tridiag(d, e)))
    x = 0.25
    want_below = int(np.sum(lam < x - 1e-12))
    got = counts(lib, d, e, x)[0]
    # x is itself an eigenvalue (of the decoupled 1 x 1 block): the count is
    # that of a point just below or just above it
    assert got in (want_below, want_below + 1)
    # a coupled example: d_0 = x exactly, the next minor is -e_0^2 (nonzero)
    d2 = np.array([0.2, 0.6, -0.4, 0.1, 0.3])
    e2 = np.array([0.5, 0.1, 0.4, 0.2])
    lam2 = np.sort(np.linalg.eigvalsh(tridiag(d2, e2)))
    assert counts(lib, d2, e2, 0.2)[0] == int(np.sum(lam2 < 0.2))


def test_decoupled_blocks(lib):
    rng = np.random.default_rng(3)
    d, e = random_unit_tridiag(rng, 40)
    e[[9, 10, 25]] = 0.0  # four blocks
    lam = np.sort(np.linalg.eigvalsh(tridiag(d, e)))
    for x in rng.uniform(-1, 1, 60):
        if np.min(np.abs(lam - x)) > 1e-10:
            assert counts(lib, d, e, x) == (int(np.sum(lam < x)),) * 2


def test_long_chains_rescale(lib):
    # p = 3000 with |d - x| up to 2: the minors overflow without rescaling;
    # and a chain with tiny |d - x| and tiny e that underflows without it
    rng = np.random.default_rng(11)
    p = 3000
    d, e = random_unit_tridiag(rng, p)
    lam = np.sort(np.linalg.eigvalsh(tridiag(d, e)))
    for x in [-1.01, -0.999, -0.5, 0.0, 0.37, 0.999, 1.01]:
        if np.min(np.abs(lam - x)) > 1e-10:
            assert counts(lib, d, e, x) == (int(np.sum(lam < x)),) * 2, x
    d3 = np.full(400, 1e-3) + 1e-9 * np.arange(400)
    e3 = np.full(399, 1e-6)
    lam3 = np.sort(np.linalg.eigvalsh(tridiag(d3, e3)))
    for x in [0.0, 0.5e-3, 1.0e-3 + 2e-7, 2e-3]:
        if np.min(np.abs(lam3 - x)) > 1e-15:
            assert counts(lib, d3, e3, x)[0] == int(np.sum(lam3 < x)), x


@pytest.mark.parametrize("kind", ["random", "interchanges"])
def test_inverse_iteration_finds_the_eigenvector(lib, kind):
    rng = np.random.default_rng(21)
    p = 120
    if kind == "random":
        d, e = random_unit_tridiag(rng, p)
    else:  # small diagonal against large off-diagonals: partial pivoting interchanges rows
        d = 1e-3 * rng.uniform(-1, 1, p)
        e = rng.uniform(0.5, 1.0, p - 1)
        s = np.abs(np.linalg.eigvalsh(tridiag(d, e))).max()
        d, e = d / s, e / s
    T = tridiag(d, e)
    lam, Q = np.linalg.eigh(T)
    for j in [0, p // 3, p - 2, p - 1]:
        if min(abs(lam[j] - lam[j - 1]) if j > 0 else 1, abs(lam[j + 1] - lam[j]) if j + 1 < p else 1) < 1e-6:
            continue
        z = np.zeros(p)
        w = np.zeros(3 * p)
        lib.h_inv_iter(_p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(e)), p, float(lam[j] + 1e-9), _p(z),
                       _p(w), j)
        assert abs(np.linalg.norm(z) - 1.0) < 1e-12
        assert abs(abs(z @ Q[:, j]) - 1.0) < 1e-10, (kind, j)
        assert np.linalg.norm(T @ z - lam[j] * z) < 1e-12
    if kind == "interchanges":  # the interchange flag rides in the multipliers' last bit
        flags = [int(np.frombuffer(np.float64(v).tobytes(), dtype=np.int64)[0] & 1) for v in w[0::3][: p - 1]]
        assert 0 < sum(flags) < p - 1


def test_device_philox_matches_the_known_answer_vectors(lib):
    path = os.path.join(HERE, "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr = (C.c_uint * 4)(*v[0:4])
        out = (C.c_uint * 4)()
        lib.h_philox(ctr, v[4], v[5], out)
        assert list(out) == v[6:10], r
