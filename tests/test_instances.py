"""The seeded synthetic inputs (paper_1912_02767_gb300/instances.py) follow
their stated recipe: the constraint maps, costs and right-hand sides of each
family, the Haar spectrum of the projection sweep with its warm start, the
batch and serving mixes, and the seeding (PCG64(1_000_003 c + i))."""
import numpy as np
import pytest

from paper_1912_02767_gb300 import instances as gen


def constraint_map(inst, X):
    """A(X)_p = sum over the entries (p, i, j, v) of v X_ii (i == j) or
    v (X_ij + X_ji) (i < j): the SDPA convention."""
    out = np.zeros(inst.m)
    for p, i, j, v in zip(inst.cp, inst.ci, inst.cj, inst.cv):
        out[p] += v * (X[i, i] if i == j else X[i, j] + X[j, i])
    return out


def random_sym(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return 0.5 * (A + A.T)


def test_seeding_is_pcg64_of_config_and_index():
    a = gen.rng_for(3, 7).random(5)
    b = np.random.Generator(np.random.PCG64(1_000_003 * 3 + 7)).random(5)
    assert np.array_equal(a, b)
    g1, g2 = gen.workload_batch(3), gen.workload_batch(3)
    assert [x.n for x in g1] == [x.n for x in g2] and np.array_equal(g1[1].C, g2[1].C)


def test_maxcut_cost_and_diagonal_constraints():
    inst = gen.maxcut(30, 0.3, np.random.default_rng(1))
    L = gen.laplacian(30, inst.meta["edges"])
    assert np.array_equal(inst.C, -0.25 * L) and np.allclose(inst.C, inst.C.T)
    assert np.allclose(L.sum(axis=1), 0.0)
    assert np.allclose(np.diag(L), np.bincount(inst.meta["edges"].ravel(), minlength=30))
    X = random_sym(30, 2)
    assert inst.m == 30 and np.allclose(constraint_map(inst, X), np.diag(X)) and np.all(inst.b == 1.0)
    # <C, x x^T> with x = +-1 is minus the cut size
    x = np.where(np.random.default_rng(3).random(30) < 0.5, -1.0, 1.0)
    cut = sum(1 for i, j in inst.meta["edges"] if x[i] != x[j])
    assert abs(x @ inst.C @ x + cut) < 1e-12


def test_theta_constraints():
    inst = gen.theta(25, 0.3, np.random.default_rng(4))
    E = inst.meta["edges"]
    assert inst.m == 1 + len(E) and np.array_equal(inst.C, -np.ones((25, 25)))
    X = random_sym(25, 5)
    ax = constraint_map(inst, X)
    assert abs(ax[0] - np.trace(X)) < 1e-12
    assert np.allclose(ax[1:], [X[i, j] for i, j in E])
    assert inst.b[0] == 1.0 and np.all(inst.b[1:] == 0.0)


def test_primal_infeasible_has_a_farkas_vector():
    inst = gen.primal_infeasible(20, 0.2, np.random.default_rng(6))
    assert inst.m == 21
    X = random_sym(20, 7)
    ax = constraint_map(inst, X)
    assert np.allclose(ax[:20], np.diag(X)) and abs(ax[20] - np.trace(X)) < 1e-12
    # y = (-1, ..., -1, 1): A^T y = 0 and b^T y = -n + n/2 < 0
    y = np.concatenate([-np.ones(20), [1.0]])
    assert abs(y @ ax) < 1e-12 and y @ inst.b == -10.0


def test_dual_infeasible_has_an_improving_ray():
    inst = gen.dual_infeasible(6)
    ray = np.zeros((6, 6))
    ray[1, 1] = 1.0
    assert constraint_map(inst, ray)[0] == 0.0 and np.sum(inst.C * ray) == -1.0


def test_haar_orthogonal_and_spectrum():
    sp = gen.random_spectrum(80, 0.1, np.random.default_rng(8))
    Q, lam, k = sp["Q"], sp["lam"], sp["k"]
    assert k == 8 and np.abs(Q.T @ Q - np.eye(80)).max() < 1e-12
    ev = np.linalg.eigvalsh(sp["W"])
    assert np.abs(np.sort(lam) - ev).max() < 1e-12
    assert np.all((lam[:k] >= 0.1) & (lam[:k] <= 1.0)) and np.all((lam[k:] >= -1.0) & (lam[k:] <= -0.1))
    # warm start: the positive eigenvectors moved by about 1e-3 per column
    d = np.linalg.norm(sp["X0"] - Q[:, :k], axis=0)
    assert 2e-4 < np.median(d) < 3e-3


@pytest.mark.parametrize("n,f", [(256, 0.01), (256, 0.25), (1024, 0.05)])
def test_projection_sweep_matrices(n, f):
    sp = gen.workload_projection(n, f)
    assert sp["W"].shape == (n, n) and sp["k"] == max(1, round(f * n))
    assert np.allclose(sp["W"], sp["W"].T)


def test_sweep_matrices_are_distinct_per_size_and_fraction():
    a, b = gen.workload_projection(256, 0.01), gen.workload_projection(256, 0.05)
    assert not np.allclose(a["Q"], b["Q"])


def test_batch_and_serving_mixes():
    batch = gen.workload_batch(40)
    assert len(batch) == 40 and all(64 <= x.n <= 1024 for x in batch)
    reqs = gen.workload_serving(400, rate=50.0, maxcut_n=(100, 150), theta_n=(100, 120))
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0) and 5.0 < t[-1] < 12.0  # 400 arrivals at 50/s
    fam = [r[1].meta["family"] for r in reqs]
    frac = {f: fam.count(f) / len(fam) for f in ("maxcut", "theta", "pinf")}
    assert 0.38 < frac["maxcut"] < 0.57 and 0.38 < frac["theta"] < 0.57 and 0.01 < frac["pinf"] < 0.10
