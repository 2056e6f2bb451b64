"""The allocation-free projection entry point, sdp_project_psd_noalloc.

It serves callers that cannot allocate device memory: code running while a
CUDA stream is being captured into a graph, where cudaMalloc is not
permitted, and applications that pool all device memory at start-up.  Its
scratch is one fixed device array shared by every call.  The test checks,
through the C ABI, that two calls in a row (same and different inputs)
agree with the closed form Pi(Q Lambda Q^T) = Q Lambda_+ Q^T and with the
allocating entry point sdp_project_psd within the FP64 projection
tolerance, that an in-place call (W is out) gives the same result, and that
sizes beyond the stated maximum are rejected.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
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


def test_noalloc_projection_matches_closed_form_and_allocating_entry_point(sdp):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    ctx = sdp.Context()
    for n, f, seed in [(40, 0.2, 1), (sdp.NOALLOC_MAX_N, 0.1, 2), (77, 0.3, 3)]:
        sp = gen.random_spectrum(n, f, np.random.default_rng(seed))
        exact = closed_form(sp)
        ref, _, _ = ctx.project_psd(sp["W"], sp["X0"], tol=1e-10)
        Wd = torch.from_numpy(np.ascontiguousarray(sp["W"])).cuda()
        nW = np.linalg.norm(sp["W"])
        for call in range(2):  # two calls in a row on the same scratch array
            out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            rc = sdp.project_psd_noalloc(Wd, out)
            assert rc == 0, sdp.status_str(rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.linalg.norm(got - exact) / nW <= TOL_FP64, (n, call)
            assert np.linalg.norm(got - ref) / nW <= TOL_FP64, (n, call)
        # in place: W is overwritten by its projection
        Wi = Wd.clone()
        assert sdp.project_psd_noalloc(Wi, Wi) == 0
        torch.cuda.synchronize()
        assert np.linalg.norm(Wi.cpu().numpy() - exact) / nW <= TOL_FP64, n


def test_noalloc_rejects_sizes_beyond_maximum(sdp):
    torch = pytest.importorskip("torch")
    n = sdp.NOALLOC_MAX_N + 1
    W = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(W)
    assert sdp.project_psd_noalloc(W, out) == -1  # SDP_E_INVALID, nothing launched
