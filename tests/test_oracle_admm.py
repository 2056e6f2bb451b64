"""Pins for the oracle's ADMM (Algorithm 1): linear step, objective values that
the mathematics fixes, and infeasibility certificates (Theorem 1, Section 5.2)."""
import itertools

import numpy as np
import pytest

from paper_1912_02767_gb300 import instances as gen


def cons_of(orc, inst):
    return orc.Constraints(inst.n, inst.m, inst.cp, inst.ci, inst.cj, inst.cv)


def _sym(n, rng):
    A = rng.standard_normal((n, n))
    return A + A.T


@pytest.mark.parametrize("family", ["maxcut", "theta", "pinf", "dense"])
def test_linear_step_matches_dense_kkt(orc, family):
    """Linear step of Algorithm 1 (Eq. kkt_system) versus a dense solve of the
    full quasidefinite KKT matrix Q in svec coordinates (independent route)."""
    rng = np.random.default_rng(1)
    n = 6
    if family == "maxcut":
        inst = gen.maxcut(n, 0.5, rng)
    elif family == "theta":
        inst = gen.theta(n, 0.5, rng)
    elif family == "pinf":
        inst = gen.primal_infeasible(n, 0.5, rng)
    else:  # random dense constraints: K has no diagonal block at all
        m = 5
        cp, ci, cj, cv = [], [], [], []
        for p in range(m):
            for i in range(n):
                for j in range(i, n):
                    cp.append(p); ci.append(i); cj.append(j); cv.append(rng.standard_normal())
        inst = gen.SDPInstance("dense", n, _sym(n, rng), m, np.array(cp), np.array(ci), np.array(cj),
                               np.array(cv), rng.standard_normal(m))
    cons = cons_of(orc, inst)
    sigma, rho = 1e-3, 0.7
    r = _sym(n, rng)
    xt = orc.linear_step(cons, n, sigma, rho, r)
    # svec coordinates: x_v = [X_ii, sqrt2 X_ij], <A,X>_F = svec(A).svec(X)
    iu = [(i, j) for j in range(n) for i in range(j + 1)]
    sc = np.array([1.0 if i == j else np.sqrt(2) for i, j in iu])
    sv = lambda M: np.array([M[i, j] for i, j in iu]) * sc
    Amat = np.zeros((inst.m, len(iu)))
    for p in range(inst.m):
        Ap = np.zeros((n, n))
        sel = inst.cp == p
        for i, j, v in zip(inst.ci[sel], inst.cj[sel], inst.cv[sel]):
            Ap[i, j] += v
            if i != j:
                Ap[j, i] += v
        Amat[p] = sv(Ap)
    Abar = np.vstack([Amat, np.eye(len(iu))])
    nv, mb = len(iu), Abar.shape[0]
    Q = np.block([[sigma * np.eye(nv), rho * Abar.T], [rho * Abar, -rho * np.eye(mb)]])
    # right-hand side chosen so that sigma x - q + rho Abar^T(z - y/rho) = r
    rhs = np.concatenate([sv(r), np.zeros(mb)])
    sol = np.linalg.solve(Q, rhs)
    Xv = sol[:nv] / sc
    Xref = np.zeros((n, n))
    for (i, j), v in zip(iu, Xv):
        Xref[i, j] = v
        Xref[j, i] = v
    assert np.allclose(xt, Xref, atol=1e-10 * max(1, np.abs(Xref).max()))


def test_kfactor_partitions(orc):
    rng = np.random.default_rng(2)
    assert orc.KFactor(cons_of(orc, gen.maxcut(10, 0.3, rng)), 1e-6, 1.0).nF == 0
    assert orc.KFactor(cons_of(orc, gen.theta(10, 0.3, rng)), 1e-6, 1.0).nF == 0
    assert orc.KFactor(cons_of(orc, gen.primal_infeasible(10, 0.3, rng)), 1e-6, 1.0).nF == 1


def _maxcut_brute(n, edges):
    best = 0
    for bits in range(1 << (n - 1)):
        s = [(bits >> i) & 1 for i in range(n)]
        best = max(best, sum(1 for i, j in edges if s[i] != s[j]))
    return best


def _solve(orc, inst, **kw):
    kw.setdefault("eps_abs", 1e-7)
    kw.setdefault("max_iter", 20000)
    kw.setdefault("check_every", 20)
    return orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, **kw)


@pytest.mark.parametrize("seed", range(4))
def test_maxcut_brute_force_bounds(orc, seed):
    """maxcut <= SDP value <= maxcut / 0.87856 (Goemans-Williamson)."""
    rng = np.random.default_rng(seed)
    n = 8 + seed
    inst = gen.maxcut(n, 0.5, rng)
    res = _solve(orc, inst)
    assert res["status_name"] == "SOLVED"
    val = -res["obj"]
    mc = _maxcut_brute(n, inst.meta["edges"])
    assert mc - 1e-4 <= val <= mc / 0.87856 + 1e-4


@pytest.mark.parametrize("n", [5, 7, 9])
def test_maxcut_odd_cycle_closed_form(orc, n):
    inst = gen.maxcut(n, 0.0, edges=gen.cycle_edges(n))
    res = _solve(orc, inst)
    assert -res["obj"] == pytest.approx(n / 2.0 * (1 + np.cos(np.pi / n)), abs=2e-5)


def test_maxcut_complete_and_bipartite(orc):
    res = _solve(orc, gen.maxcut(6, 0.0, edges=gen.complete_edges(6)))
    assert -res["obj"] == pytest.approx(36 / 4.0, abs=2e-5)
    edges = np.array([[i, j] for i in range(3) for j in range(3, 7)])
    res = _solve(orc, gen.maxcut(7, 0.0, edges=edges))
    assert -res["obj"] == pytest.approx(len(edges), abs=2e-5)


def test_theta_c5_is_sqrt5(orc):
    res = _solve(orc, gen.theta(5, 0.0, edges=gen.cycle_edges(5)))
    assert res["status_name"] == "SOLVED"
    assert -res["obj"] == pytest.approx(np.sqrt(5.0), abs=2e-5)


@pytest.mark.parametrize("n", [7, 9])
def test_theta_odd_cycle_closed_form(orc, n):
    res = _solve(orc, gen.theta(n, 0.0, edges=gen.cycle_edges(n)))
    c = np.cos(np.pi / n)
    assert -res["obj"] == pytest.approx(n * c / (1 + c), abs=2e-5)


def test_theta_complete_and_empty(orc):
    assert -_solve(orc, gen.theta(6, 0.0, edges=gen.complete_edges(6)))["obj"] == pytest.approx(1.0, abs=2e-5)
    assert -_solve(orc, gen.theta(6, 0.0, edges=np.zeros((0, 2), int)))["obj"] == pytest.approx(6.0, abs=2e-5)


def _alpha_brute(n, edges):
    adj = set(map(tuple, edges.tolist()))
    best = 0
    for r in range(n, 0, -1):
        for S in itertools.combinations(range(n), r):
            if all((min(a, b), max(a, b)) not in adj for a, b in itertools.combinations(S, 2)):
                return r
    return best


def test_theta_bipartite_equals_independence_number(orc):
    rng = np.random.default_rng(4)
    n = 9
    edges = np.array([[i, j] for i in range(4) for j in range(4, n) if rng.random() < 0.5])
    res = _solve(orc, gen.theta(n, 0.0, edges=edges))
    assert -res["obj"] == pytest.approx(_alpha_brute(n, edges), abs=5e-5)


def test_lobpcg_admm_matches_exact_admm(orc):
    """Approximate ADMM (Algorithm 1 with Algorithm 3) reaches the same optimum."""
    inst = gen.workload_maxcut64(0)
    ex = _solve(orc, inst, eps_abs=1e-5, check_every=40)
    ap = _solve(orc, inst, eps_abs=1e-5, check_every=40, use_lobpcg=1)
    assert ex["status_name"] == ap["status_name"] == "SOLVED"
    assert abs(ap["obj"] - ex["obj"]) <= 1e-4 * abs(ex["obj"])
    assert ap["n_lobpcg"] > 0.5 * ap["iters"]


def test_primal_infeasible_certificate(orc):
    """diag(X) = 1 with <I,X> = n/2 is infeasible; delta-y must satisfy
    A^T y_e + Y ~ 0, Y nsd, b^T y_e < 0 (Theorem 1 (i))."""
    rng = np.random.default_rng(8)
    n = 10
    inst = gen.primal_infeasible(n, 0.3, rng)
    res = _solve(orc, inst, eps_abs=1e-4, check_every=40)
    assert res["status_name"] == "PRIMAL_INFEASIBLE"
    ye, Yb = res["cert_e"], res["cert_X"]
    cons = cons_of(orc, inst)
    assert np.abs(orc.AT_op(cons, n, ye) + Yb).max() < 1e-4
    assert inst.b @ ye < -1e-4
    assert np.linalg.eigvalsh(Yb).max() < 1e-4
    # Farkas family: y_diag = u 1, y_tr = w with u + w >= 0 and n(u + w/2) < 0
    u, w = ye[:n].mean(), ye[n]
    assert np.allclose(ye[:n], u, atol=1e-3)
    assert u + w >= -1e-3 and n * (u + w / 2) < 0


def test_dual_infeasible_certificate(orc):
    """min <diag(0,-1,..), X> s.t. X_11 = 1 is unbounded: delta-x psd,
    A(delta-x) = 0, <C, delta-x> < 0 (Theorem 1 (ii))."""
    inst = gen.dual_infeasible(6)
    res = _solve(orc, inst, eps_abs=1e-4, check_every=40)
    assert res["status_name"] == "DUAL_INFEASIBLE"
    xb = res["cert_X"]
    assert abs(xb[0, 0]) < 1e-4
    assert np.sum(inst.C * xb) < -1e-4
    assert np.linalg.eigvalsh(xb).min() > -1e-4


def test_planted_mistakes_are_caught(orc):
    """A plausible slip in the objective's sign or the cost scaling moves the
    C5 value away from the closed form: the pins above would fail."""
    inst = gen.maxcut(5, 0.0, edges=gen.cycle_edges(5))
    good = -_solve(orc, inst)["obj"]
    bad_scale = gen.maxcut(5, 0.0, edges=gen.cycle_edges(5))
    bad_scale.C = bad_scale.C * 2  # a dropped 1/2 somewhere
    wrong = -_solve(orc, bad_scale)["obj"]
    assert abs(good - 4.5225424859) < 2e-5 and abs(wrong - 4.5225424859) > 1.0


def test_theta_complete_graph_runs_negative_mode(orc):
    """theta(K_n) = 1.  Every vertex pair is an edge, so the optimal X is
    diagonal with unit trace and the ADMM iterate W tends to the full-rank
    I/n: more than 2n/3 of its eigenvalues are positive and the mode rule of
    Section 5 selects negative mode (LOBPCG on -W, Z = W + Pi(-W)).  The
    LOBPCG-ADMM objective must equal the closed form and the exact-projection
    ADMM, and the negative branch must have carried the solve."""
    n = 40
    inst = gen.theta(n, 0.0, edges=gen.complete_edges(n))
    cons = cons_of(orc, inst)
    kw = dict(eps_abs=1e-6, rho=1.0, tol_coef=0.1, max_iter=20000)
    ex = orc.admm_solve(n, inst.C, cons, inst.b, use_lobpcg=0, **kw)
    lo = orc.admm_solve(n, inst.C, cons, inst.b, use_lobpcg=1, **kw)
    assert ex["status_name"] == lo["status_name"] == "SOLVED"
    assert lo["n_neg"] > lo["n_lobpcg"] // 2 and lo["n_neg"] > 100
    assert abs(lo["obj"] - ex["obj"]) <= 1e-4 * abs(ex["obj"])
    assert -lo["obj"] == pytest.approx(1.0, abs=1e-5)
    assert -ex["obj"] == pytest.approx(1.0, abs=1e-5)
    # the returned X is (nearly) full rank: more than 2n/3 positive eigenvalues
    assert np.sum(np.linalg.eigvalsh(lo["x"]) > 1e-3 / n) > 2 * n // 3
