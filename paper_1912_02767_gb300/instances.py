"""Seeded synthetic SDP instances and test matrices.

This module only builds problem data (graphs, cost matrices, constraint
lists, spectra); it holds none of the solver's arithmetic.  Both the CUDA
path and the CPU oracle are fed from it.

Instance i of workload c draws from numpy ``Generator(PCG64(1_000_003*c+i))``.
Families (shaped like the SDPLIB max-cut and Lovasz-theta problems the paper
solves in Section 5.1):

* max-cut relaxation:  min <C,X>  s.t. diag(X) = 1, X psd,  C = -L/4 with L
  the Laplacian of an Erdos-Renyi graph (edge (i<j) iff U < p, unit weight);
* Lovasz theta:  max <J,X>  s.t. tr X = 1, X_ij = 0 on edges, X psd
  (posed as min <-J, X>);
* primal infeasible: max-cut cost with diag(X) = 1 and <I,X> = n/2;
* dual infeasible:   min <diag(0,-1,...,-1), X>  s.t.  X_11 = 1, X psd;
* random spectrum W = Q Lambda Q^T with Haar Q for the standalone projection.

Constraint p is stored in COO form (p, i, j, v), i <= j; an off-diagonal
entry stands for both (i,j) and (j,i) (SDPA convention).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SDPInstance:
    name: str
    n: int
    C: np.ndarray          # n x n symmetric, float64
    m: int
    cp: np.ndarray         # int32 constraint index per entry
    ci: np.ndarray         # int32 row (ci <= cj)
    cj: np.ndarray         # int32 col
    cv: np.ndarray         # float64 value
    b: np.ndarray          # m, float64
    meta: dict = field(default_factory=dict)


def rng_for(config: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1_000_003 * config + index))


def erdos_renyi_edges(n: int, p: float, rng: np.random.Generator) -> np.ndarray:
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.size) < p
    return np.stack([iu[keep], ju[keep]], axis=1).astype(np.int64)


def laplacian(n: int, edges: np.ndarray) -> np.ndarray:
    L = np.zeros((n, n))
    for i, j in edges:
        L[i, j] -= 1.0
        L[j, i] -= 1.0
        L[i, i] += 1.0
        L[j, j] += 1.0
    return L


def _diag_constraints(n: int):
    idx = np.arange(n, dtype=np.int32)
    return idx.copy(), idx.copy(), idx.copy(), np.ones(n)


def maxcut(n: int, p: float, rng: np.random.Generator = None, edges=None, name="maxcut") -> SDPInstance:
    if edges is None:
        edges = erdos_renyi_edges(n, p, rng)
    C = -0.25 * laplacian(n, edges)
    cp, ci, cj, cv = _diag_constraints(n)
    return SDPInstance(name, n, C, n, cp, ci, cj, cv, np.ones(n), {"edges": edges, "family": "maxcut"})


def theta(n: int, p: float, rng: np.random.Generator = None, edges=None, name="theta") -> SDPInstance:
    if edges is None:
        edges = erdos_renyi_edges(n, p, rng)
    ne = len(edges)
    C = -np.ones((n, n))
    cp = np.concatenate([np.zeros(n, dtype=np.int32), 1 + np.arange(ne, dtype=np.int32)])
    ci = np.concatenate([np.arange(n), edges[:, 0] if ne else np.zeros(0)]).astype(np.int32)
    cj = np.concatenate([np.arange(n), edges[:, 1] if ne else np.zeros(0)]).astype(np.int32)
    cv = np.concatenate([np.ones(n), 0.5 * np.ones(ne)])
    b = np.concatenate([[1.0], np.zeros(ne)])
    return SDPInstance(name, n, C, 1 + ne, cp, ci, cj, cv, b, {"edges": edges, "family": "theta"})


def primal_infeasible(n: int, p: float, rng: np.random.Generator = None, edges=None) -> SDPInstance:
    inst = maxcut(n, p, rng, edges=edges, name="pinf")
    cp = np.concatenate([inst.cp, np.full(n, n, dtype=np.int32)])
    ci = np.concatenate([inst.ci, np.arange(n, dtype=np.int32)])
    cj = np.concatenate([inst.cj, np.arange(n, dtype=np.int32)])
    cv = np.concatenate([inst.cv, np.ones(n)])
    b = np.concatenate([np.ones(n), [n / 2.0]])
    return SDPInstance("pinf", n, inst.C, n + 1, cp, ci, cj, cv, b, {"edges": inst.meta["edges"], "family": "pinf"})


def dual_infeasible(n: int) -> SDPInstance:
    C = np.diag(np.concatenate([[0.0], -np.ones(n - 1)]))
    return SDPInstance("dinf", n, C, 1, np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32),
                       np.ones(1), np.ones(1), {"family": "dinf"})


def cycle_edges(n: int) -> np.ndarray:
    return np.array([[min(i, (i + 1) % n), max(i, (i + 1) % n)] for i in range(n)], dtype=np.int64)


def complete_edges(n: int) -> np.ndarray:
    iu, ju = np.triu_indices(n, k=1)
    return np.stack([iu, ju], axis=1).astype(np.int64)


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar orthogonal matrix: QR of a Gaussian matrix with diag(R) > 0."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def random_spectrum(n: int, frac: float, rng: np.random.Generator, warm_noise: float = 1e-3):
    """W = Q Lambda Q^T with k = round(frac*n) eigenvalues in U[0.1,1] and
    n-k in U[-1,-0.1]; warm start = the k positive eigenvectors plus
    Gaussian noise scaled so each column moves by about warm_noise."""
    k = max(1, int(round(frac * n)))
    Q = haar_orthogonal(n, rng)
    lam = np.concatenate([rng.uniform(0.1, 1.0, k), rng.uniform(-1.0, -0.1, n - k)])
    W = (Q * lam[None, :]) @ Q.T
    W = 0.5 * (W + W.T)
    X0 = Q[:, :k] + (warm_noise / np.sqrt(n)) * rng.standard_normal((n, k))
    return {"W": np.asfortranarray(W), "Q": Q, "lam": lam, "k": k, "X0": np.asfortranarray(X0)}


# ----------------------------------------------------------------------------
# Workloads (index c is the workload number used to seed the generator)
# ----------------------------------------------------------------------------
PROJ_SWEEP_N = (256, 1024, 4096)
PROJ_SWEEP_F = (0.01, 0.05, 0.25)


def workload_maxcut64(i: int = 0) -> SDPInstance:
    """Max-cut relaxation, n = 64, edge probability 0.1."""
    return maxcut(64, 0.1, rng_for(0, i), name="maxcut64")


def workload_projection(n: int, frac: float):
    """Standalone projection matrix of the sweep n in {256,1024,4096}, k/n in {1,5,25}%."""
    idx = PROJ_SWEEP_N.index(n) * len(PROJ_SWEEP_F) + PROJ_SWEEP_F.index(frac) if (
        n in PROJ_SWEEP_N and frac in PROJ_SWEEP_F) else 1000 + n
    return random_spectrum(n, frac, rng_for(1, idx))


def workload_theta500(i: int = 0) -> SDPInstance:
    """Lovasz theta, n = 500, edge probability 0.2."""
    return theta(500, 0.2, rng_for(2, i), name="theta500")


def workload_batch(count: int = 256, n_lo: int = 64, n_hi: int = 1024):
    """Uneven batch of max-cut instances, n ~ U{n_lo..n_hi}, p ~ U[0.02, 0.2]."""
    out = []
    for i in range(count):
        rng = rng_for(3, i)
        n = int(rng.integers(n_lo, n_hi + 1))
        p = float(rng.uniform(0.02, 0.2))
        out.append(maxcut(n, p, rng, name="batch%d" % i))
    return out


def workload_serving(count: int = 2000, rate: float = 50.0, maxcut_n=(100, 2000), theta_n=(100, 1000)):
    """Poisson request stream: 47.5% max-cut, 47.5% theta, 5% primal infeasible."""
    rng = rng_for(4, 0)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        u = float(rng.random())
        r2 = rng_for(4, 1 + i)
        p = float(r2.uniform(0.02, 0.2))
        if u < 0.475:
            n = int(r2.integers(maxcut_n[0], maxcut_n[1] + 1))
            inst = maxcut(n, p, r2, name="req%d" % i)
        elif u < 0.95:
            n = int(r2.integers(theta_n[0], theta_n[1] + 1))
            inst = theta(n, p, r2, name="req%d" % i)
        else:
            n = int(r2.integers(maxcut_n[0], maxcut_n[1] + 1))
            inst = primal_infeasible(n, p, r2)
        reqs.append((t, inst))
    return reqs
