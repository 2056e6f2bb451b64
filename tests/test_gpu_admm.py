"""GPU parity of the approximate-ADMM solver (Algorithm 1 with the LOBPCG
projection of Algorithm 3) through the C ABI, against the FP64 oracle:
|dobj|/|obj| <= 1e-4 at primal/dual residual 1e-4, residuals re-evaluated by
the oracle on the GPU's solution, and the Theorem 1 certificates."""
import numpy as np
import pytest

from paper_1912_02767_gb300 import instances as gen

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-4


@pytest.fixture(scope="module")
def sdp():
    from paper_1912_02767_gb300 import build_lib, sdpgpu
    build_lib.build()
    sdpgpu.load()
    return sdpgpu


def cons_of(orc, inst):
    return orc.Constraints(inst.n, inst.m, inst.cp, inst.ci, inst.cj, inst.cv)


def gpu_solve(sdp, inst, **kw):
    c = sdp.Context(**kw).setup(inst)
    res = c.solve()
    X, y, S = c.solution()
    return c, res, X, y, S


def test_maxcut64_matches_oracle(sdp, orc):
    """Max-cut relaxation, n = 64, p = 0.1, rho = 1, residual 1e-4."""
    inst = gen.workload_maxcut64(0)
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, eps_abs=1e-4)
    c, res, X, y, S = gpu_solve(sdp, inst, eps_abs=1e-4)
    assert res["status_name"] == "SOLVED" == ref["status_name"]
    assert abs(res["obj"] - ref["obj"]) <= OBJ_TOL * abs(ref["obj"])
    assert res["n_lobpcg"] > res["n_exact"]
    # residuals of the returned point, evaluated by the oracle (Y = -S)
    cons = cons_of(orc, inst)
    rp, rd, obj = orc.residuals(inst.n, inst.C, cons, inst.b, X, X, y, -S)
    assert rd <= 1e-4 + 1e-12
    assert abs(obj - res["obj"]) <= 1e-9 * abs(obj)


def test_exact_only_matches_oracle_iterates(sdp, orc):
    """Exact projection every iteration: the GPU runs the same iteration as
    the oracle, so iterations and objective agree closely."""
    inst = gen.maxcut(24, 0.3, np.random.default_rng(3))
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, eps_abs=1e-5, check_every=10)
    c, res, X, y, S = gpu_solve(sdp, inst, eps_abs=1e-5, check_every=10, exact_only=1)
    assert res["status_name"] == "SOLVED" and res["iters"] == ref["iters"]
    assert abs(res["obj"] - ref["obj"]) <= 1e-8 * abs(ref["obj"])
    assert np.abs(X - ref["x"]).max() <= 1e-7


def test_exact_syevd_comparator_matches_oracle_iterates(sdp, orc):
    """The exact-eigendecomposition comparator through the cuSOLVER syevd
    library routine (exact_solver = 1) runs the oracle's exact-projection
    iteration as closely as the built-in Jacobi does."""
    inst = gen.maxcut(24, 0.3, np.random.default_rng(3))
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, eps_abs=1e-5, check_every=10)
    c, res, X, y, S = gpu_solve(sdp, inst, eps_abs=1e-5, check_every=10, exact_only=1, exact_solver=1)
    assert res["status_name"] == "SOLVED" and res["iters"] == ref["iters"]
    assert abs(res["obj"] - ref["obj"]) <= 1e-8 * abs(ref["obj"])
    assert np.abs(X - ref["x"]).max() <= 1e-7


@pytest.mark.parametrize("seed", [0, 1])
def test_maxcut_brute_force_and_closed_forms(sdp, seed):
    rng = np.random.default_rng(seed)
    n = 10
    inst = gen.maxcut(n, 0.5, rng)
    _, res, _, _, _ = gpu_solve(sdp, inst, eps_abs=1e-6, check_every=20, max_iter=20000)
    edges = inst.meta["edges"]
    best = 0
    for bits in range(1 << (n - 1)):
        best = max(best, sum(1 for i, j in edges if ((bits >> i) & 1) != ((bits >> j) & 1)))
    assert best - 1e-3 <= -res["obj"] <= best / 0.87856 + 1e-3
    inst5 = gen.maxcut(5, 0.0, edges=gen.cycle_edges(5))
    _, r5, _, _, _ = gpu_solve(sdp, inst5, eps_abs=1e-6, check_every=20)
    assert -r5["obj"] == pytest.approx(2.5 * (1 + np.cos(np.pi / 5)), abs=5e-5)


def test_theta_c5_sqrt5(sdp):
    inst = gen.theta(5, 0.0, edges=gen.cycle_edges(5))
    _, res, _, _, _ = gpu_solve(sdp, inst, eps_abs=1e-6, check_every=20)
    assert res["status_name"] == "SOLVED"
    assert -res["obj"] == pytest.approx(np.sqrt(5.0), abs=5e-5)


def test_theta_small_matches_oracle(sdp, orc):
    """Lovasz theta, n = 40, p = 0.2, rho = 10.  Fixed-rho ADMM without scaling
    converges slowly on theta and at residual 1e-4 its objective is only
    fixed to ~1e-3 (two correct runs stopping at different points of the
    same tolerance differ by that much), so the objective is compared at
    residual 1e-6, where it is fixed well inside 1e-4."""
    inst = gen.theta(40, 0.2, np.random.default_rng(13))
    kw = dict(eps_abs=1e-6, rho=10.0, tol_coef=0.1, max_iter=40000)
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, use_lobpcg=1, **kw)
    _, res, _, _, _ = gpu_solve(sdp, inst, **kw)
    assert res["status_name"] == ref["status_name"] == "SOLVED"
    assert abs(res["obj"] - ref["obj"]) <= OBJ_TOL * abs(ref["obj"])


def test_primal_infeasible_certificate(sdp, orc):
    """diag(X) = 1 with <I,X> = n/2.  The LOBPCG tolerance constant is 0.1
    (tol = 0.1/k^1.01): with the paper's 10/k^1.01 the projection errors keep
    ||A^T y-bar|| above eps_pinf for thousands of iterations (the paper also
    reports slower convergence of this quantity with LOBPCG, Section 5.2)."""
    n = 30
    inst = gen.primal_infeasible(n, 0.2, np.random.default_rng(8))
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, eps_abs=1e-4, use_lobpcg=1, tol_coef=0.1)
    assert ref["status_name"] == "PRIMAL_INFEASIBLE"
    c, res, _, _, _ = gpu_solve(sdp, inst, eps_abs=1e-4, tol_coef=0.1)
    assert res["status_name"] == "PRIMAL_INFEASIBLE"
    ye, Yb = c.certificate()
    cons = cons_of(orc, inst)
    assert np.abs(orc.AT_op(cons, n, ye) + Yb).max() < 1e-4
    assert inst.b @ ye < -1e-4
    assert np.linalg.eigvalsh(Yb).max() < 1e-4


def test_dual_infeasible_certificate(sdp):
    inst = gen.dual_infeasible(12)
    c, res, _, _, _ = gpu_solve(sdp, inst, eps_abs=1e-4)
    assert res["status_name"] == "DUAL_INFEASIBLE"
    _, xb = c.certificate()
    assert abs(xb[0, 0]) < 1e-4
    assert np.sum(inst.C * xb) < -1e-4
    assert np.linalg.eigvalsh(xb).min() > -1e-4


def test_batch_equals_alone(sdp):
    """Instances solved together in one batched launch sequence give the same
    results as solved alone."""
    insts = [gen.maxcut(n, 0.15, np.random.default_rng(100 + n)) for n in (40, 72, 129, 64)]
    alone = [gpu_solve(sdp, inst, eps_abs=1e-4)[1] for inst in insts]
    ctxs = [sdp.Context(eps_abs=1e-4).setup(inst) for inst in insts]
    together = sdp.batch_solve(ctxs)
    for a, t in zip(alone, together):
        assert a["status_name"] == t["status_name"] == "SOLVED"
        assert a["iters"] == t["iters"]
        assert abs(a["obj"] - t["obj"]) <= 1e-9 * abs(a["obj"])


def test_server_continuous_batching(sdp):
    """Requests arriving while others run are admitted as slots free up; each
    result equals the one solved alone."""
    insts = [gen.maxcut(n, 0.2, np.random.default_rng(200 + n)) for n in (30, 50, 41, 66, 35)]
    alone = [gpu_solve(sdp, inst, eps_abs=1e-4)[1] for inst in insts]
    ctxs = [sdp.Context(eps_abs=1e-4).setup(inst) for inst in insts]
    srv = sdp.Server(budget_bytes=1 << 34, max_slots=2, iters_per_step=40, eps_abs=1e-4)
    tickets = [srv.submit(ctxs[0]), srv.submit(ctxs[1])]
    srv.step()
    tickets += [srv.submit(c) for c in ctxs[2:]]
    for _ in range(1000):
        a, q = srv.step()
        if a == 0 and q == 0:
            break
    for t, ref in zip(tickets, alone):
        rc, info = srv.poll(t)
        assert info["status"] == ref["status"] and info["iters"] == ref["iters"]
        assert abs(info["obj"] - ref["obj"]) <= 1e-9 * abs(ref["obj"])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_theta_complete_graph_negative_mode(sdp, orc, prec):
    """theta(K_n) = 1, n = 40: the iterate W tends to the full-rank I/n, so
    the Section 5 rule selects negative mode (LOBPCG on -W, Z = W + Pi(-W)).
    The GPU objective equals the closed form and the oracle's, and most
    projections ran in negative mode."""
    n = 40
    inst = gen.theta(n, 0.0, edges=gen.complete_edges(n))
    kw = dict(eps_abs=1e-6, rho=1.0, tol_coef=0.1, max_iter=20000)
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, use_lobpcg=1, **kw)
    p = sdp.PREC_FP64 if prec == "fp64" else sdp.PREC_BF16X3
    _, res, X, _, _ = gpu_solve(sdp, inst, precision=p, **kw)
    assert res["status_name"] == ref["status_name"] == "SOLVED"
    assert res["n_neg"] > res["n_lobpcg"] // 2 and res["n_neg"] > 100, res
    assert abs(res["obj"] - ref["obj"]) <= OBJ_TOL * abs(ref["obj"])
    # closed form: FP64 to the stop rule's slack; mixed to the split-BF16 product level
    assert -res["obj"] == pytest.approx(1.0, abs=1e-5 if prec == "fp64" else OBJ_TOL)


def test_maxcut64_mixed_matches_oracle(sdp, orc):
    """The mixed path (tensor-core products, FP64 Grams and Rayleigh-Ritz,
    FP64 ADMM state) on max-cut n = 64 at residual 1e-4."""
    inst = gen.workload_maxcut64(0)
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, eps_abs=1e-4)
    c, res, X, y, S = gpu_solve(sdp, inst, eps_abs=1e-4, precision=sdp.PREC_BF16X3)
    assert res["status_name"] == "SOLVED" == ref["status_name"]
    assert abs(res["obj"] - ref["obj"]) <= OBJ_TOL * abs(ref["obj"])
    assert res["n_lobpcg"] > res["n_exact"]
    rp, rd, obj = orc.residuals(inst.n, inst.C, cons_of(orc, inst), inst.b, X, X, y, -S)
    assert rd <= 1e-4 + 1e-12


def test_theta_small_mixed_matches_oracle(sdp, orc):
    """Lovasz theta n = 40 on the mixed path, compared at residual 1e-6 as in
    the FP64 test."""
    inst = gen.theta(40, 0.2, np.random.default_rng(13))
    kw = dict(eps_abs=1e-6, rho=10.0, tol_coef=0.1, max_iter=40000)
    ref = orc.admm_solve(inst.n, inst.C, cons_of(orc, inst), inst.b, use_lobpcg=1, **kw)
    _, res, _, _, _ = gpu_solve(sdp, inst, precision=sdp.PREC_BF16X3, **kw)
    assert res["status_name"] == ref["status_name"] == "SOLVED"
    assert abs(res["obj"] - ref["obj"]) <= OBJ_TOL * abs(ref["obj"])


def test_batch_mixed_matches_oracle_objectives(sdp):
    """An uneven max-cut batch (n ~ U{64..256}) solved together on the mixed
    path: each instance's objective against the FP64 oracle's LOBPCG-ADMM
    objective stored by tests/golden/make_batch_objectives.py."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "batch_maxcut_objectives.json")))
    insts = gen.workload_batch(len(gold["instances"]), 64, 256)
    ctxs = [sdp.Context(eps_abs=1e-4, precision=sdp.PREC_BF16X3).setup(i) for i in insts]
    infos = sdp.batch_solve(ctxs)
    solved = 0
    for g, inst, r in zip(gold["instances"], insts, infos):
        assert inst.n == g["n"]
        if g["status"] == "SOLVED":
            assert r["status_name"] == "SOLVED", (g, r)
            assert abs(r["obj"] - g["obj"]) <= OBJ_TOL * abs(g["obj"]), (g, r)
            solved += 1
        else:  # the oracle itself stops at the iteration limit (slow fixed-rho ADMM)
            assert r["status_name"] in ("MAX_ITER", "SOLVED"), (g, r)
    assert solved >= len(gold["instances"]) // 2
