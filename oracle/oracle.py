"""ctypes front-end of the plain FP64 CPU oracle (oracle/sdp_oracle.c).

TEST INFRASTRUCTURE ONLY.  Each function states which part of the paper
(Rontsis, Goulart, Nakatsukasa, "Efficient Semidefinite Programming with
approximate ADMM") it follows; the C file holds the arithmetic.

Conventions: dense matrices are numpy float64 arrays, column-major
(Fortran order) when passed to C.  A constraint set is given in COO form
(cp, ci, cj, cv) with ci <= cj; an off-diagonal entry v of constraint p
stands for both (i,j) and (j,i), so <A_p, X> counts it twice.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB, build

_lib = None

ORC_SOLVED, ORC_PRIMAL_INFEASIBLE, ORC_DUAL_INFEASIBLE, ORC_MAX_ITER = 1, 2, 3, 4
STATUS_NAMES = {0: "OK", 1: "SOLVED", 2: "PRIMAL_INFEASIBLE", 3: "DUAL_INFEASIBLE", 4: "MAX_ITER",
                -1: "E_INVALID", -2: "E_NOMEM", -4: "E_NUMERICAL"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Cons(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("nnz", C.c_long),
                ("cp", _ip), ("ci", _ip), ("cj", _ip), ("cv", _dp)]


class _Settings(C.Structure):
    _fields_ = [("rho", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double),
                ("eps_abs", C.c_double), ("eps_rel", C.c_double), ("eps_pinf", C.c_double),
                ("eps_dinf", C.c_double), ("max_iter", C.c_int), ("check_every", C.c_int),
                ("use_lobpcg", C.c_int), ("lobpcg_maxit", C.c_int), ("tol_coef", C.c_double),
                ("tol_exp", C.c_double), ("expand_frac", C.c_double), ("mode_frac", C.c_double),
                ("seed", C.c_uint64)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("obj", C.c_double), ("r_prim", C.c_double),
                ("r_dual", C.c_double), ("n_exact", C.c_int), ("n_lobpcg", C.c_int),
                ("lobpcg_steps", C.c_int), ("expansions", C.c_int), ("last_rank", C.c_int),
                ("n_neg", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        L = C.CDLL(LIB)
        L.orc_philox4x32.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_normal.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_normal.restype = C.c_double
        L.orc_jacobi_eig.argtypes = [C.c_int, _dp, _dp, _dp]
        L.orc_psd_project.argtypes = [C.c_int, _dp, _dp, _ip, _ip]
        L.orc_cholesky.argtypes = [C.c_int, _dp, _dp]
        L.orc_is_pd_shifted.argtypes = [C.c_int, _dp, C.c_double]
        L.orc_A.argtypes = [C.POINTER(_Cons), _dp, _dp]
        L.orc_AT_add.argtypes = [C.POINTER(_Cons), _dp, C.c_double, _dp]
        L.orc_linear_step.argtypes = [C.POINTER(_Cons), C.c_double, C.c_double, _dp, _dp]
        L.orc_kfactor.argtypes = [C.POINTER(_Cons), C.c_double, C.c_double]
        L.orc_kfactor.restype = C.c_void_p
        L.orc_kfactor_nF.argtypes = [C.c_void_p]
        L.orc_ksolve.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_kfree.argtypes = [C.c_void_p]
        L.orc_rayleigh_ritz.argtypes = [C.c_int, _dp, C.c_int, _dp, _dp, _dp]
        L.orc_lobpcg.argtypes = [C.c_int, _dp, _ip, C.c_int, _dp, _dp, C.c_double, C.c_int, C.c_int,
                                 C.c_uint64, C.c_uint32, _ip, _dp]
        L.orc_lobpcg_project.argtypes = [C.c_int, _dp, _ip, C.c_int, _dp, C.c_double, C.c_int, _dp, _ip]
        L.orc_admm_solve.argtypes = [C.c_int, _dp, C.POINTER(_Cons), _dp, C.POINTER(_Settings),
                                     _dp, _dp, _dp, _dp, _dp, C.POINTER(_Info)]
        _lib = L
    return _lib


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Constraints:
    """Keeps the COO arrays alive while C holds pointers into them."""

    def __init__(self, n, m, cp, ci, cj, cv):
        self.cp = np.ascontiguousarray(cp, dtype=np.int32)
        self.ci = np.ascontiguousarray(ci, dtype=np.int32)
        self.cj = np.ascontiguousarray(cj, dtype=np.int32)
        self.cv = np.ascontiguousarray(cv, dtype=np.float64)
        if np.any(self.ci > self.cj):
            raise ValueError("COO entries must have i <= j")
        self.s = _Cons(int(n), int(m), int(self.cp.size), self.cp.ctypes.data_as(_ip), self.ci.ctypes.data_as(_ip),
                       self.cj.ctypes.data_as(_ip), _ptr(self.cv))


def philox4x32(counter, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32(c, k, o)
    return [int(v) for v in o]


def normal(seed, stream, draw, row, col):
    return lib().orc_normal(seed, stream, draw, row, col)


def jacobi_eig(A):
    """Full eigendecomposition by cyclic Jacobi: (lam ascending, V, sweeps)."""
    A = _f64(A)
    n = A.shape[0]
    lam = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sw = lib().orc_jacobi_eig(n, _ptr(A), _ptr(lam), _ptr(V))
    if sw < 0:
        raise RuntimeError("Jacobi did not converge")
    return lam, V, sw


def psd_project(A):
    """Pi_{S+}(A) by full eigendecomposition (Eq. 2): (P, npos, nneg)."""
    A = _f64(A)
    n = A.shape[0]
    out = np.zeros((n, n), order="F")
    npos, nneg = C.c_int(), C.c_int()
    rc = lib().orc_psd_project(n, _ptr(A), _ptr(out), C.byref(npos), C.byref(nneg))
    if rc:
        raise RuntimeError("projection failed")
    return out, npos.value, nneg.value


def cholesky(A):
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros((n, n), order="F")
    bad = lib().orc_cholesky(n, _ptr(A), _ptr(L))
    return L, bad


def is_pd_shifted(M, shift):
    M = _f64(M)
    return bool(lib().orc_is_pd_shifted(M.shape[0], _ptr(M), shift))


def A_op(cons: Constraints, n, X):
    X = _f64(X)
    u = np.zeros(cons.s.m)
    lib().orc_A(C.byref(cons.s), _ptr(X), _ptr(u))
    return u


def AT_op(cons: Constraints, n, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    X = np.zeros((n, n), order="F")
    lib().orc_AT_add(C.byref(cons.s), _ptr(u), 1.0, _ptr(X))
    return X


def linear_step(cons: Constraints, n, sigma, rho, r):
    """x~ = ((sigma+rho) I + rho A^T A)^{-1} r (linear step of Algorithm 1)."""
    r = _f64(r)
    xt = np.zeros((n, n), order="F")
    rc = lib().orc_linear_step(C.byref(cons.s), sigma, rho, _ptr(r), _ptr(xt))
    if rc:
        raise RuntimeError("K factorisation failed")
    return xt


class KFactor:
    def __init__(self, cons: Constraints, sigma, rho):
        self.cons = cons
        self.h = lib().orc_kfactor(C.byref(cons.s), sigma, rho)
        if not self.h:
            raise RuntimeError("K factorisation failed")
        self.nF = lib().orc_kfactor_nF(self.h)

    def solve(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.zeros_like(u)
        lib().orc_ksolve(self.h, _ptr(u), _ptr(v))
        return v

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_kfree(self.h)
            self.h = None


def rayleigh_ritz(A, S):
    """Algorithm 2: Ritz vectors and values (ascending) of A on span(S)."""
    A = _f64(A)
    S = _f64(S)
    n, p = S.shape
    V = np.zeros((n, p), order="F")
    lam = np.zeros(p)
    rc = lib().orc_rayleigh_ritz(n, _ptr(A), p, _ptr(S), _ptr(V), _ptr(lam))
    if rc:
        raise RuntimeError("Cholesky QR breakdown")
    return lam, V


def lobpcg(A, X0, tol, maxit=20, bexp=None, mcap=None, seed=0, stream=0):
    """Algorithm 3 (positive eigenpairs).  Returns dict with X, lam, resn, info."""
    A = _f64(A)
    n = A.shape[0]
    m = X0.shape[1]
    if bexp is None:
        bexp = max(1, int(np.ceil(n / 50)))
    if mcap is None:
        mcap = n
    X = np.zeros((n, mcap), order="F")
    X[:, :m] = X0
    lam = np.zeros(mcap)
    resn = np.zeros(mcap)
    info = (C.c_int * 4)()
    mm = C.c_int(m)
    rc = lib().orc_lobpcg(n, _ptr(A), C.byref(mm), mcap, _ptr(X), _ptr(lam), tol, maxit, bexp, seed, stream,
                          info, _ptr(resn))
    m = mm.value
    return {"rc": rc, "X": np.array(X[:, :m]), "lam": lam[:m].copy(), "resn": resn[:m].copy(), "m": m,
            "rr_steps": info[0], "expansions": info[1], "converged": bool(info[2]), "npos": info[3]}


def lobpcg_project(A, X0, tol, maxit=20, mcap=None):
    """Pi_{S+}(A) by LOBPCG (Algorithm 3) from the warm block X0 and the
    reconstruction of Eq. 2, all in the C oracle (one thread).  Returns
    (P, info dict)."""
    A = _f64(A)
    n = A.shape[0]
    m = X0.shape[1]
    if mcap is None:
        mcap = n
    X = np.zeros((n, mcap), order="F")
    X[:, :m] = X0
    out = np.zeros((n, n), order="F")
    info = (C.c_int * 4)()
    mm = C.c_int(m)
    rc = lib().orc_lobpcg_project(n, _ptr(A), C.byref(mm), mcap, _ptr(X), tol, maxit, _ptr(out), info)
    return out, {"rc": rc, "m": mm.value, "rr_steps": info[0], "expansions": info[1], "converged": bool(info[2]),
                 "npos": info[3]}


def default_settings(**kw):
    s = dict(rho=1.0, sigma=1e-6, alpha=1.6, eps_abs=1e-4, eps_rel=0.0, eps_pinf=1e-4, eps_dinf=1e-4,
             max_iter=5000, check_every=40, use_lobpcg=0, lobpcg_maxit=20, tol_coef=10.0, tol_exp=1.01,
             expand_frac=1.0 / 50.0, mode_frac=1.0 / 3.0, seed=0)
    s.update(kw)
    return s


def admm_solve(n, C_mat, cons: Constraints, b, **settings):
    """Algorithm 1 on min <C,X> s.t. A(X) = b, X psd (exact or LOBPCG projection)."""
    st = default_settings(**settings)
    S = _Settings(**{k: st[k] for k, _ in _Settings._fields_})
    Cm = _f64(C_mat)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = cons.s.m
    x = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    Y = np.zeros((n, n), order="F")
    ye = np.zeros(m)
    cert = np.zeros(m + n * n)
    info = _Info()
    rc = lib().orc_admm_solve(n, _ptr(Cm), C.byref(cons.s), _ptr(b), C.byref(S), _ptr(x), _ptr(Z), _ptr(Y),
                              _ptr(ye), _ptr(cert), C.byref(info))
    out = {f: getattr(info, f) for f, _ in _Info._fields_}
    out.update(rc=rc, status_name=STATUS_NAMES.get(info.status, str(info.status)), x=x, Z=Z, Y=Y, ye=ye,
               cert_e=cert[:m].copy(), cert_X=cert[m:].reshape((n, n), order="F").copy())
    return out


def residuals(n, C_mat, cons: Constraints, b, x, Z, ye, Y):
    """Primal/dual residuals and objective of a given iterate (Algorithm 1 form (P))."""
    Ax = A_op(cons, n, x)
    r_prim = max(np.max(np.abs(Ax - b)) if b.size else 0.0, np.max(np.abs(x - Z)))
    r_dual = np.max(np.abs(np.asarray(C_mat) + AT_op(cons, n, ye) + Y))
    obj = float(np.sum(np.asarray(C_mat) * x))
    return r_prim, r_dual, obj
