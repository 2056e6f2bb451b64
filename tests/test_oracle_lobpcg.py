"""Pins for the oracle's Rayleigh-Ritz (Algorithm 2) and LOBPCG (Algorithm 3),
and the projection error bound of Theorem 3."""
import numpy as np
import pytest

from paper_1912_02767_gb300 import instances as gen


def test_rayleigh_ritz_exact_on_invariant_subspace(orc):
    """RR on a span of eigenvectors returns those eigenpairs exactly."""
    rng = np.random.default_rng(0)
    sp = gen.random_spectrum(40, 0.2, rng)
    Q, lam = sp["Q"], sp["lam"]
    cols = [0, 3, 5]
    S = Q[:, cols] @ rng.standard_normal((3, 3))  # same span, not orthonormal
    th, V = orc.rayleigh_ritz(sp["W"], S)
    assert np.allclose(th, np.sort(lam[cols]), atol=1e-13)
    assert np.linalg.norm(sp["W"] @ V - V * th) < 1e-12


def test_rayleigh_ritz_interlacing(orc):
    """Cauchy interlacing: the i-th largest Ritz value <= i-th largest eigenvalue."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 30))
    A = A + A.T
    S = rng.standard_normal((30, 6))
    th, _ = orc.rayleigh_ritz(A, S)
    ev = np.sort(np.linalg.eigvalsh(A))
    assert np.all(th[::-1] <= ev[::-1][:6] + 1e-12)
    assert np.all(th >= ev[:6] - 1e-12)


@pytest.mark.parametrize("n,f", [(60, 0.05), (100, 0.1), (128, 0.25)])
def test_lobpcg_converges_to_exact_projection(orc, n, f):
    rng = np.random.default_rng(n)
    sp = gen.random_spectrum(n, f, rng, warm_noise=1e-2)
    res = orc.lobpcg(sp["W"], sp["X0"], tol=1e-11, maxit=50)
    assert res["rc"] == 0 and res["converged"]
    pos = res["lam"] > 0
    P = (res["X"][:, pos] * res["lam"][pos]) @ res["X"][:, pos].T
    Pref = (sp["Q"] * np.maximum(sp["lam"], 0)) @ sp["Q"].T
    assert np.linalg.norm(P - Pref) <= 1e-9 * np.linalg.norm(sp["W"])
    assert res["npos"] == sp["k"]


def test_lobpcg_expansion_finds_missing_eigenpairs(orc):
    """A block that starts with fewer columns than positive eigenvalues must
    expand with random columns (the expansion step of Algorithm 3) and still end exact."""
    rng = np.random.default_rng(3)
    n, k = 80, 12
    sp = gen.random_spectrum(n, k / n, rng)
    X0 = rng.standard_normal((n, 4))  # 4 columns for 12 positive eigenvalues
    res = orc.lobpcg(sp["W"], X0, tol=1e-10, maxit=200, bexp=4, mcap=40, seed=9)
    assert res["rc"] == 0 and res["converged"]
    assert res["expansions"] >= 1 and res["m"] >= k
    pos = res["lam"] > 0
    P = (res["X"][:, pos] * res["lam"][pos]) @ res["X"][:, pos].T
    Pref = (sp["Q"] * np.maximum(sp["lam"], 0)) @ sp["Q"].T
    assert np.linalg.norm(P - Pref) <= 1e-8 * np.linalg.norm(sp["W"])


def test_lobpcg_capacity_exceeded_is_reported(orc):
    rng = np.random.default_rng(4)
    sp = gen.random_spectrum(60, 0.5, rng)
    res = orc.lobpcg(sp["W"], rng.standard_normal((60, 2)), tol=1e-10, maxit=100, bexp=2, mcap=6)
    assert res["rc"] == -2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_theorem3_bound_holds(orc, seed):
    """||V L V^T - Pi(A)||_F^2 <= 2||R||_F^2 + ||Pi(V_perp^T A V_perp)||_F^2 for
    Ritz pairs (Theorem 3) -- checked on loose, unconverged LOBPCG output."""
    rng = np.random.default_rng(50 + seed)
    n = 70
    sp = gen.random_spectrum(n, 0.1, rng, warm_noise=0.3)
    res = orc.lobpcg(sp["W"], sp["X0"], tol=1e-1, maxit=1)
    V, th = res["X"], res["lam"]
    pos = th > 0
    Vp, thp = V[:, pos], th[pos]
    approx = (Vp * thp) @ Vp.T
    exact = (sp["Q"] * np.maximum(sp["lam"], 0)) @ sp["Q"].T
    R = sp["W"] @ Vp - Vp * thp
    # orthonormal complement of span(Vp) by a library QR (independent route)
    Qf, _ = np.linalg.qr(np.hstack([Vp, rng.standard_normal((n, n - Vp.shape[1]))]))
    Vperp = Qf[:, Vp.shape[1]:]
    B = Vperp.T @ sp["W"] @ Vperp
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    perp = np.sum(np.maximum(ev, 0) ** 2)
    lhs = np.linalg.norm(approx - exact) ** 2
    assert lhs <= 2 * np.linalg.norm(R) ** 2 + perp + 1e-12


def test_negative_mode_reconstruction_is_the_projection(orc):
    """Negative mode (Section 5): with more than 2n/3 positive eigenvalues the
    projection is computed from the positive eigenpairs of -W, Pi(W) = W +
    Pi(-W) (Eq. 2's second form).  LOBPCG on -W from a perturbed block of
    W's negative eigenvectors, then the reconstruction, must give the closed
    form Q Lambda_+ Q^T (k/n = 0.8); the Moreau decomposition W = Pi(W) -
    Pi(-W) then holds.  A sign slip (reconstructing from -W) is caught."""
    rng = np.random.default_rng(11)
    n, k = 90, 72
    sp = gen.random_spectrum(n, k / n, rng)
    W, Q, lam = sp["W"], sp["Q"], sp["lam"]
    neg = np.where(lam < 0)[0]
    X0 = Q[:, neg] + 1e-3 / np.sqrt(n) * rng.standard_normal((n, neg.size))
    res = orc.lobpcg(-W, X0, tol=1e-11, maxit=50)
    assert res["rc"] == 0 and res["converged"] and res["npos"] == n - k
    pos = res["lam"] > 0
    Pneg = (res["X"][:, pos] * res["lam"][pos]) @ res["X"][:, pos].T   # Pi(-W)
    Z = W + Pneg
    exact = (Q * np.maximum(lam, 0)) @ Q.T
    nW = np.linalg.norm(W)
    assert np.linalg.norm(Z - exact) <= 1e-9 * nW
    assert np.linalg.norm((Z - Pneg) - W) <= 1e-12 * nW                 # Moreau: Pi(W) - Pi(-W) = W
    assert np.linalg.eigvalsh(Z).min() >= -1e-9 and np.linalg.eigvalsh(-Pneg).max() <= 1e-9
    planted = -W + Pneg                                                 # sign slip in the reconstruction
    assert np.linalg.norm(planted - exact) > 1e-2 * nW


@pytest.mark.parametrize("n,f", [(80, 0.05), (120, 0.25)])
def test_lobpcg_projection_matches_closed_form(orc, n, f):
    """The oracle's standalone LOBPCG projection (Algorithm 3 + Eq. 2) from a
    warm start perturbed by 1e-3 equals Q Lambda_+ Q^T; a reconstruction that
    kept the negative Ritz values too would return W itself instead."""
    sp = gen.random_spectrum(n, f, np.random.default_rng(900 + n))
    nW = np.linalg.norm(sp["W"])
    P, info = orc.lobpcg_project(sp["W"], sp["X0"], tol=1e-10)
    assert info["rc"] == 0 and info["converged"] and info["npos"] == sp["k"]
    exact = (sp["Q"] * np.maximum(sp["lam"], 0)) @ sp["Q"].T
    assert np.linalg.norm(P - exact) <= 1e-8 * nW
    assert np.linalg.norm(sp["W"] - exact) > 0.1 * nW
