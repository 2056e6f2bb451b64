"""GPU parity of the PSD projection (Eq. 2) computed by LOBPCG (Algorithm 3)
through the C ABI, against the closed form Pi(Q Lambda Q^T) = Q Lambda_+ Q^T
and against the oracle's Jacobi projection.  FP64 mode: ||dPi||_F/||W||_F
<= 1e-6."""
import numpy as np
import pytest

from paper_1912_02767_gb300 import instances as gen

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-6


@pytest.fixture(scope="module")
def sdp():
    from paper_1912_02767_gb300 import build_lib, sdpgpu
    build_lib.build()
    sdpgpu.load()
    return sdpgpu


def closed_form(sp):
    return (sp["Q"] * np.maximum(sp["lam"], 0)) @ sp["Q"].T


@pytest.mark.parametrize("n,f", [(40, 0.1), (64, 0.05), (100, 0.2), (257, 0.03), (300, 0.3)])
def test_projection_matches_closed_form_and_oracle(sdp, orc, n, f):
    sp = gen.random_spectrum(n, f, np.random.default_rng(n))
    ctx = sdp.Context()
    P, V, info = ctx.project_psd(sp["W"], sp["X0"])
    ref = closed_form(sp)
    nW = np.linalg.norm(sp["W"])
    assert np.linalg.norm(P - ref) / nW <= TOL_FP64
    Pj, _, _ = orc.psd_project(sp["W"])
    assert np.linalg.norm(P - Pj) / nW <= TOL_FP64
    assert info["npos"] == sp["k"]
    # Theorem 3: ||Pi~ - Pi||_F <= sqrt(2) ||R_+||_F (+ perp term, zero here)
    assert np.linalg.norm(P - ref) <= np.sqrt(2) * info["res_fro"] + 1e-10 * nW


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("n,f", [(300, 0.3), (1024, 0.1)])
def test_projection_soft_locking(sdp, n, f, prec):
    """Soft locking (converged pairs leave R and dX) narrows the trial
    subspace but reaches the same projection; (1024, 0.1) runs the cluster
    tridiagonalization (p about 300)."""
    sp = gen.random_spectrum(n, f, np.random.default_rng(n + 7))
    p = sdp.PREC_FP64 if prec == "fp64" else sdp.PREC_BF16X3
    ctx = sdp.Context(precision=p, soft_lock=1)
    P, V, info = ctx.project_psd(sp["W"], sp["X0"])
    err = np.linalg.norm(P - closed_form(sp)) / np.linalg.norm(sp["W"])
    assert err <= (TOL_FP64 if prec == "fp64" else 1e-4), err
    assert info["npos"] == sp["k"]


def test_projection_expands_block(sdp):
    """Start with 3 random columns for 12 positive eigenvalues: the block must
    grow by random columns (Algorithm 3, expansion) and still be exact."""
    n, k = 120, 12
    sp = gen.random_spectrum(n, k / n, np.random.default_rng(5))
    X0 = np.random.default_rng(6).standard_normal((n, 3))
    ctx = sdp.Context(lobpcg_max_iter=200)
    P, V, info = ctx.project_psd(sp["W"], X0, tol=1e-9)
    assert info["expansions"] >= 1 and info["m"] >= k
    assert np.linalg.norm(P - closed_form(sp)) / np.linalg.norm(sp["W"]) <= TOL_FP64


def test_projection_host_and_device_paths_agree(sdp):
    torch = pytest.importorskip("torch")
    n = 130
    sp = gen.random_spectrum(n, 0.05, np.random.default_rng(9))
    ctx = sdp.Context()
    P_h, V_h, _ = ctx.project_psd(sp["W"], sp["X0"], tol=1e-10)
    Wd = torch.from_numpy(np.ascontiguousarray(sp["W"])).cuda()
    Xd = torch.from_numpy(np.ascontiguousarray(sp["X0"])).cuda()
    P_d, V_d, _ = ctx.project_psd(Wd, Xd, tol=1e-10, on_device=True)
    assert np.abs(P_d.cpu().numpy() - P_h).max() <= 1e-12 * np.abs(P_h).max()


def test_projection_degenerate_cases(sdp):
    ctx = sdp.Context()
    # negative definite: projection is zero
    n = 50
    rng = np.random.default_rng(1)
    Q = gen.haar_orthogonal(n, rng)
    W = (Q * -rng.uniform(0.1, 1, n)) @ Q.T
    P, V, info = ctx.project_psd(W, rng.standard_normal((n, 2)), tol=1e-10)
    assert np.abs(P).max() <= 1e-9 and info["npos"] == 0
    # n = 1 and repeated positive eigenvalues
    P1, _, _ = ctx.project_psd(np.array([[2.5]]), np.array([[1.0]]), tol=1e-12)
    assert abs(P1[0, 0] - 2.5) < 1e-12
    lam = np.array([1.0] * 4 + [-1.0] * (n - 4))
    W = (Q * lam) @ Q.T
    P, V, info = ctx.project_psd(W, Q[:, :4] + 1e-3 * rng.standard_normal((n, 4)), tol=1e-10)
    assert np.linalg.norm(P - (Q[:, :4] @ Q[:, :4].T)) <= 1e-8


@pytest.mark.parametrize("n,f", [(256, 0.01), (256, 0.05), (256, 0.25), (1024, 0.01), (1024, 0.05)])
def test_projection_sweep_sizes(sdp, n, f):
    """Projection-sweep matrices (Haar Q, spectrum U[0.1,1] / U[-1,-0.1],
    warm start perturbed by 1e-3) at full size against the closed form."""
    sp = gen.workload_projection(n, f)
    ctx = sdp.Context()
    P, V, info = ctx.project_psd(sp["W"], sp["X0"])
    assert np.linalg.norm(P - closed_form(sp)) / np.linalg.norm(sp["W"]) <= TOL_FP64


@pytest.mark.parametrize("n,f", [(300, 0.2), (1024, 0.05)])
def test_projection_mixed_precision(sdp, n, f):
    """Mixed path (split-BF16 x3 products on the tensor cores, FP32 Grams,
    FP64 Rayleigh-Ritz and residual norms): the error against the closed
    form is bounded by the FP32 level."""
    sp = gen.random_spectrum(n, f, np.random.default_rng(77 + n))
    ctx = sdp.Context(precision=sdp.PREC_BF16X3)
    nW = np.linalg.norm(sp["W"])
    P, V, info = ctx.project_psd(sp["W"], sp["X0"], tol=1e-5 * nW / np.sqrt(2 * sp["k"]))
    err = np.linalg.norm(P - closed_form(sp)) / nW
    assert err <= 1e-4, err
    assert info["npos"] == sp["k"]


@pytest.mark.parametrize("n,k", [(64, 8), (200, 37), (1024, 51), (1000, 300), (4096, 205)])
def test_block_product_tensor_cores(sdp, n, k):
    """W B on the tcgen05 tensor cores (split-BF16 x3, FP32 accumulation)
    against an FP64 product: relative error at the bf16-split level; FP64
    mode exact to rounding.  Sizes span several 128-row tiles, ragged
    tails, N tiles up to 256 and split-K."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n + k)
    A = rng.standard_normal((n, n))
    W = 0.5 * (A + A.T)
    B = rng.standard_normal((n, k))
    ref = W @ B
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()   # column-major n x k
    for prec, tol in [(sdp.PREC_FP64, 1e-13), (sdp.PREC_BF16X3, 3e-5)]:
        ctx = sdp.Context(precision=prec)
        out = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda")
        ctx.block_product(Wd, Bd, out)
        got = out.cpu().numpy().T
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert np.all(np.isfinite(got)) and err <= tol, (prec, err)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("n,f", [(100, 0.2), (257, 0.03), (300, 0.3)])
def test_rayleigh_ritz_methods_agree(sdp, n, f, prec):
    """The Rayleigh-Ritz step by tridiagonal reduction (Householder, Sturm
    bisection, inverse iteration) and by cyclic Jacobi both give the
    projection of Eq. 2 at the precision's level, with the same rank."""
    sp = gen.random_spectrum(n, f, np.random.default_rng(500 + n))
    nW = np.linalg.norm(sp["W"])
    ref = closed_form(sp)
    p = sdp.PREC_FP64 if prec == "fp64" else sdp.PREC_BF16X3
    tol = None if prec == "fp64" else 1e-5 * nW / np.sqrt(2 * sp["k"])
    bound = TOL_FP64 if prec == "fp64" else 1e-4
    out = []
    for rm in (0, 1):
        ctx = sdp.Context(precision=p, rr_method=rm)
        P, V, info = ctx.project_psd(sp["W"], sp["X0"]) if tol is None else ctx.project_psd(sp["W"], sp["X0"], tol=tol)
        assert np.linalg.norm(P - ref) / nW <= bound, (rm, np.linalg.norm(P - ref) / nW)
        assert info["npos"] == sp["k"]
        out.append(P)
    assert np.linalg.norm(out[0] - out[1]) / nW <= 2 * bound


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_projection_repeated_eigenvalues(sdp, prec):
    """Eigenvalues repeated exactly (multiplicities 8 and 4 among the
    positives, 20 at -1): the Ritz block is any orthonormal basis of each
    eigenspace and the projection is still exact."""
    n = 160
    rng = np.random.default_rng(21)
    Q = gen.haar_orthogonal(n, rng)
    lam = np.concatenate([np.full(8, 1.0), np.full(4, 0.5), np.full(20, -1.0), -rng.uniform(0.1, 0.9, n - 32)])
    W = (Q * lam) @ Q.T
    X0 = Q[:, :12] + 1e-3 * rng.standard_normal((n, 12))
    ref = (Q[:, :12] * lam[:12]) @ Q[:, :12].T
    p = sdp.PREC_FP64 if prec == "fp64" else sdp.PREC_BF16X3
    ctx = sdp.Context(precision=p)
    tol = 1e-10 if prec == "fp64" else 1e-5 * np.linalg.norm(W) / np.sqrt(24)
    P, V, info = ctx.project_psd(W, X0, tol=tol)
    assert info["npos"] == 12
    assert np.linalg.norm(P - ref) / np.linalg.norm(W) <= (TOL_FP64 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_projection_negative_mode(sdp, prec):
    """Negative mode (Section 5, Eq. 2's second form): W with k/n = 0.8
    positive eigenvalues; the warm block approximates the eigenvectors of the
    negative ones, LOBPCG runs on -W (the products take alpha = -1) and the
    reconstruction is Z = W + Pi(-W).  Closed form at the precision's level."""
    n, k = 300, 240
    rng = np.random.default_rng(801)
    sp = gen.random_spectrum(n, k / n, rng)
    Q, lam = sp["Q"], sp["lam"]
    neg = np.where(lam < 0)[0]
    X0 = Q[:, neg] + 1e-3 / np.sqrt(n) * rng.standard_normal((n, neg.size))
    nW = np.linalg.norm(sp["W"])
    p = sdp.PREC_FP64 if prec == "fp64" else sdp.PREC_BF16X3
    ctx = sdp.Context(precision=p, proj_neg=1)
    tol = 0.0 if prec == "fp64" else 1e-5 * nW / np.sqrt(2 * neg.size)
    P, V, info = ctx.project_psd(sp["W"], X0, tol=tol)
    err = np.linalg.norm(P - closed_form(sp)) / nW
    assert info["mode"] == 1 and info["npos"] == n - k, info
    assert err <= (TOL_FP64 if prec == "fp64" else 1e-4), err


@pytest.mark.parametrize("n,f", [(1024, 0.25), (4096, 0.01), (4096, 0.05), (4096, 0.25)])
def test_projection_sweep_full_size_fp64(sdp, n, f):
    """The sweep's largest matrices in FP64 mode (products, Grams and
    Rayleigh-Ritz FP64) against the closed form at 1e-6."""
    sp = gen.workload_projection(n, f)
    ctx = sdp.Context()
    P, V, info = ctx.project_psd(sp["W"], sp["X0"])
    assert np.linalg.norm(P - closed_form(sp)) / np.linalg.norm(sp["W"]) <= TOL_FP64
    assert info["npos"] == sp["k"]


@pytest.mark.parametrize("n,f", [(1024, 0.25), (4096, 0.25)])
def test_projection_sweep_full_size_mixed(sdp, n, f):
    """The same matrices on the mixed path (tensor-core products, FP64
    Grams and Rayleigh-Ritz): the closed-form error stays at the split-BF16
    product level."""
    sp = gen.workload_projection(n, f)
    nW = np.linalg.norm(sp["W"])
    ctx = sdp.Context(precision=sdp.PREC_BF16X3)
    P, V, info = ctx.project_psd(sp["W"], sp["X0"], tol=1e-5 * nW / np.sqrt(2 * sp["k"]))
    assert np.linalg.norm(P - closed_form(sp)) / nW <= 1e-4
    assert info["npos"] == sp["k"]


def test_bounded_waits_give_up_and_the_context_stays_usable(sdp):
    """A bounded device wait that reaches its limit gives up: the call
    returns SDP_E_TIMEOUT (no trap, no hang) and, with the default limit
    restored, the same context computes correctly.  Covered: the tcgen05
    pipeline waits of the block product and the grid barriers of the
    cooperative Rayleigh-Ritz kernels."""
    torch = pytest.importorskip("torch")
    n, k = 1024, 64
    rng = np.random.default_rng(3)
    A = rng.standard_normal((n, n))
    W = 0.5 * (A + A.T)
    B = rng.standard_normal((n, k))
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    ctx = sdp.Context(precision=sdp.PREC_BF16X3)
    out = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    try:
        assert sdp.set_wait_limit(1e-9) == 0
        with pytest.raises(RuntimeError, match="E_TIMEOUT"):
            ctx.block_product(Wd, Bd, out)
        # a wide trial subspace: Rayleigh-Ritz on the whole GPU (grid barriers)
        sp = gen.random_spectrum(600, 1 / 3, np.random.default_rng(4))
        pctx = sdp.Context()
        with pytest.raises(RuntimeError, match="E_TIMEOUT"):
            pctx.project_psd(sp["W"], sp["X0"])
    finally:
        sdp.set_wait_limit(0.0)
    ctx.block_product(Wd, Bd, out)
    torch.cuda.synchronize()
    ref = W @ B
    assert np.linalg.norm(out.cpu().numpy().T - ref) / np.linalg.norm(ref) <= 3e-5
    P, _, info = pctx.project_psd(sp["W"], sp["X0"])
    assert np.linalg.norm(P - closed_form(sp)) / np.linalg.norm(sp["W"]) <= TOL_FP64
    assert sdp.set_wait_limit(-1.0) == -1
