"""The FP64-accurate tensor-core product (sdp_dense_product): the split-
product GEMM that the mixed-precision Rayleigh-Ritz step (Algorithm 2 inside
Algorithm 3) uses for its Grams, H = L^{-1} M L^{-T}, Ritz coefficients and
block update.  Checked through the C ABI against an FP64 product within the
stated bound |dC| <= K 2^-44 max|a_m.| max|b_.n| (+ FP64 rounding of the
reference), bit-exactly on integer data whose product FP64 holds exactly
(every digit product and every 128-deep chunk sum is exact), across tile
edges, ragged tails, split-K, all four transpose combinations, beta != 0
and non-finite inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdp():
    from paper_1912_02767_gb300 import build_lib, sdpgpu
    build_lib.build()
    sdpgpu.load()
    return sdpgpu


def _dev(torch, X):
    """column-major device copy of a numpy matrix (torch shape = X.T)"""
    return torch.from_numpy(np.ascontiguousarray(X.T)).cuda()


def _run(sdp, torch, A, B, ta, tb, alpha=1.0, beta=0.0, C0=None):
    M = A.shape[1] if ta else A.shape[0]
    N = B.shape[0] if tb else B.shape[1]
    Cd = _dev(torch, C0 if C0 is not None else np.full((M, N), np.nan if beta == 0.0 else 0.0))
    ctx = sdp.Context(precision=sdp.PREC_BF16X3)
    ctx.dense_product(_dev(torch, A), _dev(torch, B), Cd, trans_a=ta, trans_b=tb, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    return Cd.cpu().numpy().T


@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (200, 70, 300), (1000, 333, 4096), (37, 5, 1000), (513, 129, 65)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_dense_product_within_bound(sdp, M, N, K, ta, tb):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    opA = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))   # rows of very different scale
    opB = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    A = opA.T.copy() if ta else opA
    B = opB.T.copy() if tb else opB
    got = _run(sdp, torch, A, B, ta, tb, alpha=0.75)
    ref = 0.75 * (opA @ opB)
    bound = 0.75 * K * 2.0 ** -44 * np.abs(opA).max(1)[:, None] * np.abs(opB).max(0)[None, :]
    bound += 8 * K * 2.0 ** -53 * (np.abs(opA) @ np.abs(opB)) + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


def test_dense_product_exact_on_integer_data(sdp):
    """Integer entries below 2^10, K = 4096: op(A) op(B) is exact in FP64 and
    so is the split product (a few leading digits per entry, every chunk sum
    below 2^24): bit-exact, split-K included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    for M, N, K in [(300, 200, 4096), (64, 64, 128), (129, 65, 4097)]:
        A = rng.integers(-1023, 1024, (M, K)).astype(np.float64)
        B = rng.integers(-1023, 1024, (K, N)).astype(np.float64)
        got = _run(sdp, torch, A, B, False, False)
        assert np.array_equal(got, A @ B), (M, N, K)


def test_dense_product_beta_and_nonfinite(sdp):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    M, N, K = 150, 90, 260
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C0 = rng.standard_normal((M, N))
    got = _run(sdp, torch, A, B, False, False, alpha=-1.0, beta=0.5, C0=C0)
    ref = -(A @ B) + 0.5 * C0
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    A[3, 17] = np.nan
    B[5, 40] = np.inf
    got = _run(sdp, torch, A, B, False, False)
    bad = np.zeros((M, N), bool)
    bad[3, :] = True
    bad[:, 40] = True
    assert np.all(np.isnan(got[bad])) and np.all(np.isfinite(got[~bad]))


def test_dense_product_rejects_bad_arguments(sdp):
    torch = pytest.importorskip("torch")
    ctx = sdp.Context(precision=sdp.PREC_BF16X3)
    L = sdp.load()
    assert L.sdp_dense_product(ctx.h, 0, 0, -1, 2, 2, 1.0, None, 1, None, 1, 0.0, None, 1) == -1
    X = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    p = sdp._vp(X)
    assert L.sdp_dense_product(ctx.h, 0, 0, 4, 4, 4, 1.0, p, 2, p, 4, 0.0, p, 4) == -1  # lda < M
