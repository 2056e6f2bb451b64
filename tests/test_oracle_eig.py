"""Pins for the oracle's eigendecomposition and projection (Section 1, Eqs. 1-2).

Each pin is something the mathematics fixes independently of the oracle:
closed forms, invariants and known spectra.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def _haar(n, rng):
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def test_jacobi_diagonal(orc):
    d = np.array([3.0, -1.0, 0.0, 2.5, -7.0])
    lam, V, _ = orc.jacobi_eig(np.diag(d))
    assert np.array_equal(lam, np.sort(d))
    assert np.allclose(np.abs(V), np.eye(5)[:, np.argsort(d)])


@pytest.mark.parametrize("a,b,c", [(2.0, 1.0, 2.0), (1.0, -3.0, 5.0), (0.0, 1e-9, 0.0), (-4.0, 2.0, 1.0)])
def test_jacobi_2x2_closed_form(orc, a, b, c):
    lam, V, _ = orc.jacobi_eig(np.array([[a, b], [b, c]]))
    h = np.sqrt(((a - c) / 2.0) ** 2 + b * b)
    assert lam[0] == pytest.approx((a + c) / 2.0 - h, abs=1e-14)
    assert lam[1] == pytest.approx((a + c) / 2.0 + h, abs=1e-14)


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_jacobi_known_spectrum(orc, n):
    rng = np.random.default_rng(n)
    Q = _haar(n, rng)
    lam0 = np.sort(rng.uniform(-3, 3, n))
    A = (Q * lam0) @ Q.T
    A = 0.5 * (A + A.T)
    lam, V, _ = orc.jacobi_eig(A)
    assert np.allclose(lam, lam0, atol=1e-12 * max(1, n))
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.linalg.norm(A @ V - V * lam) <= 1e-12 * max(1.0, np.linalg.norm(A))


def test_jacobi_repeated_eigenvalues(orc):
    rng = np.random.default_rng(5)
    Q = _haar(12, rng)
    lam0 = np.array([1.0] * 5 + [-2.0] * 4 + [0.0] * 3)
    A = (Q * lam0) @ Q.T
    lam, V, _ = orc.jacobi_eig(A)
    assert np.allclose(lam, np.sort(lam0), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(12), atol=1e-13)


def test_jacobi_matches_library_eigh(orc):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 40))
    A = A + A.T
    lam, _, _ = orc.jacobi_eig(A)
    assert np.allclose(lam, np.linalg.eigvalsh(A), atol=1e-12)


def test_projection_of_diagonal(orc):
    d = np.array([1.5, -2.0, 0.0, 3.0, -0.1])
    P, npos, nneg = orc.psd_project(np.diag(d))
    assert np.allclose(P, np.diag(np.maximum(d, 0)), atol=1e-15)
    assert (npos, nneg) == (2, 2)


@pytest.mark.parametrize("n,k", [(16, 3), (50, 1), (50, 49), (64, 20)])
def test_projection_closed_form(orc, n, k):
    """Pi(Q Lambda Q^T) = Q Lambda_+ Q^T (Eq. 2) with no eigensolver on the right."""
    rng = np.random.default_rng(100 + n + k)
    Q = _haar(n, rng)
    lam = np.concatenate([rng.uniform(0.1, 1, k), rng.uniform(-1, -0.1, n - k)])
    W = (Q * lam) @ Q.T
    W = 0.5 * (W + W.T)
    P, npos, nneg = orc.psd_project(W)
    Pref = (Q * np.maximum(lam, 0)) @ Q.T
    assert np.linalg.norm(P - Pref) <= 1e-13 * np.linalg.norm(W)
    assert npos == k and nneg == n - k


def test_projection_moreau_invariants(orc):
    """Pi(W) psd, W - Pi(W) nsd, <Pi(W), W - Pi(W)> = 0, idempotent, W = Pi(W) - Pi(-W)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((30, 30))
    W = A + A.T
    P, _, _ = orc.psd_project(W)
    Pm, _, _ = orc.psd_project(-W)
    assert np.linalg.eigvalsh(P).min() >= -1e-12
    assert np.linalg.eigvalsh(W - P).max() <= 1e-12
    assert abs(np.sum(P * (W - P))) <= 1e-11 * np.linalg.norm(W) ** 2
    PP, _, _ = orc.psd_project(P)
    assert np.linalg.norm(PP - P) <= 1e-12 * np.linalg.norm(P)
    assert np.linalg.norm(W - (P - Pm)) <= 1e-12 * np.linalg.norm(W)


def test_cholesky_and_pd_test(orc):
    rng = np.random.default_rng(3)
    B = rng.standard_normal((10, 10))
    A = B @ B.T + 0.1 * np.eye(10)
    L, bad = orc.cholesky(A)
    assert bad == 0
    assert np.allclose(L @ L.T, A, atol=1e-12)
    assert np.allclose(L, np.linalg.cholesky(A), atol=1e-12)
    # indefinite: fails; the shift test is exact about lambda_min
    M = np.diag([1.0, 2.0, -0.5])
    assert orc.cholesky(M)[1] == 3
    assert not orc.is_pd_shifted(M, 0.4)
    assert orc.is_pd_shifted(M, 0.6)


def test_philox_known_answers(orc):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        assert orc.philox4x32(vals[0:4], vals[4:6]) == vals[6:10]


def test_normal_generator_moments(orc):
    z = np.array([orc.normal(1234, 7, 0, i, j) for i in range(200) for j in range(20)])
    assert abs(z.mean()) < 0.06 and abs(z.std() - 1.0) < 0.05
    # counter-based: same coordinates give the same number, others differ
    assert orc.normal(1, 2, 3, 4, 5) == orc.normal(1, 2, 3, 4, 5)
    assert orc.normal(1, 2, 3, 4, 5) != orc.normal(1, 2, 3, 5, 4)
