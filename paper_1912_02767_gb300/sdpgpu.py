"""Thin ctypes binding of libsdpgpu (include/sdpgpu.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Host arrays are numpy float64/int32 arrays; device arrays are
torch CUDA tensors (their data pointers are passed with the call's
on-device flag).  Loading fails loudly when the library has not been
built; there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdpgpu.so")

SDP_OK, SDP_SOLVED, SDP_PRIMAL_INFEASIBLE, SDP_DUAL_INFEASIBLE, SDP_MAX_ITER = 0, 1, 2, 3, 4
SDP_RUNNING, SDP_QUEUED = 5, 6
PREC_FP64, PREC_BF16X3, PREC_AUTO = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Settings(C.Structure):
    _fields_ = [("rho", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double), ("eps_abs", C.c_double),
                ("eps_rel", C.c_double), ("eps_pinf", C.c_double), ("eps_dinf", C.c_double),
                ("max_iter", C.c_int), ("check_every", C.c_int), ("lobpcg_max_iter", C.c_int),
                ("precision", C.c_int), ("exact_only", C.c_int), ("tol_coef", C.c_double),
                ("tol_exp", C.c_double), ("expand_frac", C.c_double), ("mode_frac", C.c_double),
                ("seed", C.c_ulonglong), ("rr_method", C.c_int), ("rr_fp32", C.c_int), ("proj_neg", C.c_int),
                ("exact_solver", C.c_int), ("soft_lock", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("obj", C.c_double), ("r_prim", C.c_double),
                ("r_dual", C.c_double), ("n_exact", C.c_int), ("n_lobpcg", C.c_int), ("lobpcg_steps", C.c_int),
                ("expansions", C.c_int), ("rank", C.c_int), ("solve_ms", C.c_double), ("n_neg", C.c_int),
                ("n_ladder", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProjInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("steps", C.c_int), ("m", C.c_int), ("npos", C.c_int),
                ("expansions", C.c_int), ("converged", C.c_int), ("res_fro", C.c_double),
                ("jacobi_sweeps", C.c_int), ("mode", C.c_int), ("fp64_products", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProfEntry(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("ms", C.c_double), ("timed", C.c_longlong), ("flops", C.c_double),
                ("bytes", C.c_double)]


PROF_FAMILIES = ["product", "gram", "rayleigh_ritz", "update", "recon", "resid", "admm", "exact", "check", "split"]

_lib = None


def load():
    """Load libsdpgpu.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsdpgpu.so is not built; run paper_1912_02767_gb300/build_lib.py "
                           "(or __graft_entry__.build()) first")
    L = C.CDLL(LIB_PATH)
    L.sdp_default_settings.argtypes = [C.POINTER(Settings)]
    L.sdp_default_settings.restype = None
    L.sdp_status_str.argtypes = [C.c_int]
    L.sdp_status_str.restype = C.c_char_p
    L.sdp_last_error.restype = C.c_char_p
    L.sdp_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Settings), C.c_void_p]
    L.sdp_setup.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_long, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_int]
    L.sdp_update_settings.argtypes = [C.c_void_p, C.POINTER(Settings)]
    L.sdp_solve.argtypes = [C.c_void_p, C.POINTER(Info)]
    L.sdp_get_solution.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.sdp_get_certificate.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.sdp_project_psd.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, _ip, C.c_int,
                                  C.c_double, C.c_int, C.POINTER(ProjInfo)]
    L.sdp_batch_solve.argtypes = [C.c_int, C.POINTER(C.c_void_p), C.POINTER(Info)]
    L.sdp_footprint_bytes.argtypes = [C.c_int, C.c_int, C.c_long, C.c_int]
    L.sdp_footprint_bytes.restype = C.c_ulonglong
    L.sdp_destroy.argtypes = [C.c_void_p]
    L.sdp_destroy.restype = None
    L.sdp_server_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Settings), C.c_ulonglong, C.c_int, C.c_int,
                                    C.c_void_p]
    L.sdp_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_ulonglong)]
    L.sdp_server_step.argtypes = [C.c_void_p, _ip, _ip]
    L.sdp_server_poll.argtypes = [C.c_void_p, C.c_ulonglong, C.POINTER(Info)]
    L.sdp_server_destroy.argtypes = [C.c_void_p]
    L.sdp_server_destroy.restype = None
    L.sdp_block_product.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    L.sdp_project_psd_noalloc.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.sdp_set_wait_limit.argtypes = [C.c_double]
    L.sdp_dense_product.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                    C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_int]
    L.sdp_prof_enable.argtypes = [C.c_int]
    L.sdp_prof_enable.restype = None
    L.sdp_prof_reset.restype = None
    L.sdp_prof_get.argtypes = [C.c_int, C.POINTER(ProfEntry)]
    L.sdp_prof_named.argtypes = [C.c_int, C.c_char_p, C.c_int, C.POINTER(ProfEntry)]
    _lib = L
    return L


def prof_enable(on=True):
    load().sdp_prof_enable(1 if on else 0)


def prof_reset():
    load().sdp_prof_reset()


def prof_get():
    """Per kernel family: launches, timed event ms, algorithmic flops and bytes."""
    L = load()
    out = {}
    for f, name in enumerate(PROF_FAMILIES):
        e = ProfEntry()
        _check(L.sdp_prof_get(f, C.byref(e)), "sdp_prof_get")
        out[name] = {"launches": e.launches, "ms": e.ms, "timed": e.timed, "flops": e.flops, "bytes": e.bytes}
    return out


def set_wait_limit(seconds):
    """sdp_set_wait_limit: limit of every bounded device wait (0 = default)."""
    return load().sdp_set_wait_limit(float(seconds))


def prof_named():
    """Per named kernel: launches, timed event ms, algorithmic flops and bytes."""
    L = load()
    out = {}
    buf = C.create_string_buffer(128)
    idx = 0
    while True:
        e = ProfEntry()
        if L.sdp_prof_named(idx, buf, 128, C.byref(e)) != 0:
            break
        out[buf.value.decode()] = {"launches": e.launches, "ms": e.ms, "timed": e.timed, "flops": e.flops,
                                   "bytes": e.bytes}
        idx += 1
    return out


def status_str(code):
    return load().sdp_status_str(code).decode()


def last_error():
    return load().sdp_last_error().decode()


def settings(**kw):
    s = Settings()
    load().sdp_default_settings(C.byref(s))
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    return s


def _check(rc, what):
    if rc < 0:
        raise RuntimeError("%s failed: %s (%s)" % (what, status_str(rc), last_error()))
    return rc


def _host_ptr(a, dtype):
    return a.ctypes.data_as(C.c_void_p)


def _vp(t):
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """One SDP instance: sdp_create + sdp_setup (+ solve / project)."""

    def __init__(self, stream=None, **kw):
        self.lib = load()
        self.h = C.c_void_p()
        self.settings = settings(**kw)
        self._keep = []
        _check(self.lib.sdp_create(C.byref(self.h), C.byref(self.settings), _stream_handle(stream)), "sdp_create")
        self.n = 0
        self.m = 0

    def setup(self, inst):
        """Load an instance with fields n, C, m, cp, ci, cj, cv, b (host arrays)."""
        n, m = int(inst.n), int(inst.m)
        Cm = np.asfortranarray(inst.C, dtype=np.float64)
        cp = np.ascontiguousarray(inst.cp, dtype=np.int32)
        ci = np.ascontiguousarray(inst.ci, dtype=np.int32)
        cj = np.ascontiguousarray(inst.cj, dtype=np.int32)
        cv = np.ascontiguousarray(inst.cv, dtype=np.float64)
        b = np.ascontiguousarray(inst.b, dtype=np.float64)
        rc = self.lib.sdp_setup(self.h, n, _host_ptr(Cm, 0), m, cp.size, _host_ptr(cp, 0), _host_ptr(ci, 0),
                                _host_ptr(cj, 0), _host_ptr(cv, 0), _host_ptr(b, 0), 0)
        _check(rc, "sdp_setup")
        self.n, self.m = n, m
        return self

    def update_settings(self, **kw):
        for k, v in kw.items():
            setattr(self.settings, k, v)
        _check(self.lib.sdp_update_settings(self.h, C.byref(self.settings)), "sdp_update_settings")

    def solve(self):
        info = Info()
        rc = _check(self.lib.sdp_solve(self.h, C.byref(info)), "sdp_solve")
        d = info.as_dict()
        d["status_name"] = status_str(info.status)
        d["rc"] = rc
        return d

    def solution(self):
        X = np.zeros((self.n, self.n), order="F")
        y = np.zeros(max(self.m, 1))
        S = np.zeros((self.n, self.n), order="F")
        _check(self.lib.sdp_get_solution(self.h, _host_ptr(X, 0), _host_ptr(y, 0), _host_ptr(S, 0), 0),
               "sdp_get_solution")
        return X, y[: self.m], S

    def certificate(self):
        cy = np.zeros(max(self.m, 1))
        cM = np.zeros((self.n, self.n), order="F")
        _check(self.lib.sdp_get_certificate(self.h, _host_ptr(cy, 0), _host_ptr(cM, 0), 0), "sdp_get_certificate")
        return cy[: self.m], cM

    def project_psd(self, W, V, tol=0.0, mcap=None, on_device=False):
        """Pi_{S+}(W) from warm start V (n x m).  numpy (host) or torch CUDA tensors
        (on_device=True).  Returns (P, V_out, info)."""
        n = W.shape[0]
        m = V.shape[1]
        if mcap is None:
            mcap = n
        mm = C.c_int(m)
        info = ProjInfo()
        if on_device:
            import torch
            out = torch.empty((n, n), dtype=torch.float64, device=W.device)
            Vbuf = torch.zeros((mcap, n), dtype=torch.float64, device=W.device)  # column-major n x mcap
            Vbuf[:m] = V.t()
            rc = self.lib.sdp_project_psd(self.h, n, C.c_void_p(W.data_ptr()), C.c_void_p(out.data_ptr()),
                                          C.c_void_p(Vbuf.data_ptr()), C.byref(mm), mcap, tol, 1, C.byref(info))
            _check(rc, "sdp_project_psd")
            return out.t(), Vbuf[: mm.value].t(), info.as_dict()
        Wf = np.asfortranarray(W, dtype=np.float64)
        out = np.zeros((n, n), order="F")
        Vbuf = np.zeros((n, mcap), order="F")
        Vbuf[:, :m] = V
        rc = self.lib.sdp_project_psd(self.h, n, _host_ptr(Wf, 0), _host_ptr(out, 0), _host_ptr(Vbuf, 0),
                                      C.byref(mm), mcap, tol, 0, C.byref(info))
        _check(rc, "sdp_project_psd")
        return out, np.array(Vbuf[:, : mm.value]), info.as_dict()

    def block_product(self, W, B, out, resplit_w=True):
        """out = W B (torch CUDA float64 tensors; W symmetric n x n, B and out
        column-major n x k, i.e. torch shape (k, n))."""
        n = W.shape[0]
        k = B.shape[0]
        _check(self.lib.sdp_block_product(self.h, n, C.c_void_p(W.data_ptr()), C.c_void_p(B.data_ptr()), k,
                                          C.c_void_p(out.data_ptr()), 1 if resplit_w else 0), "sdp_block_product")

    def dense_product(self, A, B, C, trans_a=False, trans_b=False, alpha=1.0, beta=0.0):
        """sdp_dense_product on torch CUDA float64 tensors holding column-major
        matrices: a column-major R x Q matrix is a contiguous torch tensor of
        shape (Q, R).  C = alpha op(A) op(B) + beta C, FP64-accurate on the
        tensor cores."""
        Ar, Ac = A.shape[1], A.shape[0]
        Br, Bc = B.shape[1], B.shape[0]
        M, K = (Ac, Ar) if trans_a else (Ar, Ac)
        Kb, N = (Bc, Br) if trans_b else (Br, Bc)
        assert K == Kb and C.shape[1] == M and C.shape[0] == N
        _check(self.lib.sdp_dense_product(self.h, 1 if trans_a else 0, 1 if trans_b else 0, M, N, K, float(alpha),
                                          _vp(A), max(1, Ar), _vp(B),
                                          max(1, Br), float(beta), _vp(C), max(1, M)), "sdp_dense_product")

    def project_raw(self, n, W_ptr, out_ptr, V_ptr, m, mcap, tol, on_device):
        """sdp_project_psd on raw pointers (column-major n x n W and out,
        n x mcap V holding the m warm-start columns).  Returns ProjInfo dict."""
        mm = C.c_int(m)
        info = ProjInfo()
        rc = self.lib.sdp_project_psd(self.h, n, C.c_void_p(W_ptr), C.c_void_p(out_ptr), C.c_void_p(V_ptr),
                                      C.byref(mm), mcap, tol, 1 if on_device else 0, C.byref(info))
        _check(rc, "sdp_project_psd")
        d = info.as_dict()
        d["m"] = mm.value
        return d

    def close(self):
        if self.h:
            self.lib.sdp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(ctxs):
    """Solve several set-up contexts in one batched launch sequence."""
    L = load()
    arr = (C.c_void_p * len(ctxs))(*[c.h.value for c in ctxs])
    infos = (Info * len(ctxs))()
    _check(L.sdp_batch_solve(len(ctxs), arr, infos), "sdp_batch_solve")
    out = []
    for k in range(len(ctxs)):
        d = infos[k].as_dict()
        d["status_name"] = status_str(infos[k].status)
        out.append(d)
    return out


class Server:
    """Continuous-batching server (sdp_server_*)."""

    def __init__(self, budget_bytes, max_slots=64, iters_per_step=40, stream=None, **kw):
        self.lib = load()
        self.h = C.c_void_p()
        self.settings = settings(**kw)
        _check(self.lib.sdp_server_create(C.byref(self.h), C.byref(self.settings), budget_bytes, max_slots,
                                          iters_per_step, _stream_handle(stream)), "sdp_server_create")

    def submit(self, ctx):
        t = C.c_ulonglong()
        _check(self.lib.sdp_server_submit(self.h, ctx.h, C.byref(t)), "sdp_server_submit")
        return t.value

    def step(self):
        a, q = C.c_int(), C.c_int()
        _check(self.lib.sdp_server_step(self.h, C.byref(a), C.byref(q)), "sdp_server_step")
        return a.value, q.value

    def poll(self, ticket):
        info = Info()
        rc = _check(self.lib.sdp_server_poll(self.h, ticket, C.byref(info)), "sdp_server_poll")
        d = info.as_dict()
        d["status_name"] = status_str(rc)
        return rc, d

    def close(self):
        if self.h:
            self.lib.sdp_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_N = 128


def project_psd_noalloc(W, out, stream=None):
    """sdp_project_psd_noalloc on torch CUDA tensors (n x n, float64,
    contiguous; W symmetric).  Asynchronous on `stream`; returns the status."""
    n = W.shape[0]
    return load().sdp_project_psd_noalloc(n, C.c_void_p(W.data_ptr()), C.c_void_p(out.data_ptr()),
                                          _stream_handle(stream))


def footprint_bytes(n, m, nnz, precision=PREC_FP64):
    return int(load().sdp_footprint_bytes(n, m, nnz, precision))
