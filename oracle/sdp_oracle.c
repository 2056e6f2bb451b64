/*
 * sdp_oracle.c -- plain, slow FP64 CPU oracle for approximate-ADMM
 * semidefinite programming (Rontsis, Goulart, Nakatsukasa,
 * "Efficient Semidefinite Programming with approximate ADMM").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header or table with
 * the CUDA library.
 *
 * Every routine is the textbook definition of what it computes, written in
 * the paper's order and notation, in double precision, single-threaded:
 *
 *   orc_jacobi_eig     full symmetric eigendecomposition by cyclic Jacobi
 *                      (Golub & Van Loan, Alg. 8.5.2/8.5.3); the paper's
 *                      "exact" projection uses a full eigendecomposition
 *                      (Section 1, Eq. 2).
 *   orc_psd_project    Pi_{S+}(A) = V+ Lambda+ V+^T  (Section 1, Eq. 2).
 *   orc_cholesky       dense Cholesky; a failed pivot means "not positive
 *                      definite" (cone tests, Section 5, COSMO footnote).
 *   orc_A / orc_AT     the linear map A(X)_p = <A_p, X>_F and its adjoint.
 *   orc_kfactor/solve  the linear step of Algorithm 1 (Eq. kkt_system),
 *                      after eliminating z~ = [A; I] x~: a Woodbury solve
 *                      with K = (sigma+rho) I_m + rho A A^T, K eliminated
 *                      by block Gaussian elimination (diagonal block +
 *                      dense Schur complement, Cholesky of the latter).
 *   orc_rayleigh_ritz  Algorithm 2 (orthonormalise by Cholesky QR,
 *                      eigendecomposition of S^T A S, Ritz vectors S W~).
 *   orc_lobpcg         Algorithm 3 (positive eigenpairs, expansion by
 *                      b random columns when more than m Ritz values of
 *                      the trial subspace are positive).
 *   orc_admm_solve     Algorithm 1 on  min <C,X>  s.t.  A(X) = b, X psd,
 *                      cast in form (P) with P = 0, q = C, A-bar = [A; I],
 *                      cone {b} x S+, with exact or LOBPCG projections,
 *                      the positive/negative/exact mode rule of Section 5,
 *                      and the infeasibility tests of Section 5.2
 *                      (Theorem 1 certificates).
 *   orc_philox4x32     Philox4x32-10 counter-based generator (Salmon et
 *                      al., SC'11), used for the random expansion columns
 *                      so that both implementations draw identical numbers.
 *
 * Readings of the paper (where it is silent or garbled) are fixed here and
 * repeated in the design notes:
 *   - the dual update of Algorithm 1 is read as y <- y + rho(alpha z~ + (1-alpha) z - z+),
 *     so Y+ = rho (W - Pi(W)) and y_e+ = rho (w_e - b).
 *   - Eq. at the end of Section 4 "Pi = I - V- Lambda- V-^T" is read as
 *     A - V- Lambda- V-^T (Eq. 2).
 *   - Matrices use the Frobenius inner product (svec with sqrt(2) scaling).
 *   - Infeasibility: S_C(y) read as b^T y_e < -eps_pinf with Y <= 0 tested
 *     by Cholesky of (-Y + eps I); dual test <C, x> < -eps_dinf with
 *     A(x) ~ 0 and x + eps I positive definite.  Normalisation by inf-norm.
 *   - LOBPCG stops when every Ritz pair of the block has ||r_i||_2 <= tol
 *     (the rule of the experiments, Section 5; a rule on the positive pairs
 *     alone is vacuous when the block holds no positive Ritz value);
 *     convergence is checked before each Rayleigh-Ritz step.
 *
 * Matrices are dense, column-major, leading dimension n.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_SOLVED 1
#define ORC_PRIMAL_INFEASIBLE 2
#define ORC_DUAL_INFEASIBLE 3
#define ORC_MAX_ITER 4
#define ORC_E_INVALID (-1)
#define ORC_E_NOMEM (-2)
#define ORC_E_NUMERICAL (-4)

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC 2011).                                      */
/* ------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One standard normal deviate for element (row, col) of the random block
 * drawn at draw number `draw` of stream `stream`: counter = (row, col, draw,
 * stream), key = seed.  Two 53-bit uniforms from the four output words, then
 * Box-Muller (cosine branch). */
double orc_normal(uint64_t seed, uint32_t stream, uint32_t draw, uint32_t row, uint32_t col) {
  uint32_t ctr[4] = {row, col, draw, stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32(ctr, key, o);
  uint64_t a = (((uint64_t)o[0] << 32) | o[1]) >> 11;
  uint64_t b = (((uint64_t)o[2] << 32) | o[3]) >> 11;
  double u1 = ((double)a + 1.0) * (1.0 / 9007199254740992.0); /* (0,1] */
  double u2 = (double)b * (1.0 / 9007199254740992.0);         /* [0,1) */
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* ------------------------------------------------------------------ */
/* Small dense helpers                                                 */
/* ------------------------------------------------------------------ */
static double* dalloc(size_t count) { return (double*)calloc(count ? count : 1, sizeof(double)); }

/* C (r x c) = A^T B with A (k x r), B (k x c), all column-major with ld = rows */
static void gemm_tn(int k, int r, int c, const double* A, const double* B, double* C) {
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < r; ++i) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[IDX(t, i, k)] * B[IDX(t, j, k)];
      C[IDX(i, j, r)] = s;
    }
}

/* C (r x c) = A (r x k) B (k x c) */
static void gemm_nn(int r, int k, int c, const double* A, const double* B, double* C) {
  for (int j = 0; j < c; ++j) {
    for (int i = 0; i < r; ++i) C[IDX(i, j, r)] = 0.0;
    for (int t = 0; t < k; ++t) {
      double b = B[IDX(t, j, k)];
      for (int i = 0; i < r; ++i) C[IDX(i, j, r)] += A[IDX(i, t, r)] * b;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Cyclic Jacobi eigendecomposition (Golub & Van Loan, Section 8.5).   */
/* lam ascending; V columns are the matching orthonormal eigenvectors. */
/* Stops when off(A) <= 1e-15 ||A||_F or a sweep rotates nothing.      */
/* Returns the number of sweeps, or -1 if 100 sweeps did not converge. */
/* ------------------------------------------------------------------ */
int orc_jacobi_eig(int n, const double* A_in, double* lam, double* V) {
  if (n <= 0) return 0;
  double* A = dalloc((size_t)n * n);
  memcpy(A, A_in, sizeof(double) * (size_t)n * n);
  /* symmetrise the input (use the average of both triangles) */
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) {
      double v = 0.5 * (A[IDX(i, j, n)] + A[IDX(j, i, n)]);
      A[IDX(i, j, n)] = v;
      A[IDX(j, i, n)] = v;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (size_t t = 0; t < (size_t)n * n; ++t) fro += A[t] * A[t];
  fro = sqrt(fro);
  int sweeps = 0, converged = (fro == 0.0);
  while (!converged && sweeps < 100) {
    double off = 0.0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        if (i != j) off += A[IDX(i, j, n)] * A[IDX(i, j, n)];
    off = sqrt(off);
    if (off <= 1e-15 * fro) { converged = 1; break; }
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[IDX(p, q, n)];
        double app = A[IDX(p, p, n)], aqq = A[IDX(q, q, n)];
        if (apq == 0.0) continue;
        if (fabs(apq) <= 1e-18 * (fabs(app) + fabs(aqq))) {
          A[IDX(p, q, n)] = 0.0;
          A[IDX(q, p, n)] = 0.0;
          continue;
        }
        /* symmetric Schur decomposition of the 2x2 block (GVL Alg 8.5.2) */
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* A <- A J (columns p, q) */
        for (int k = 0; k < n; ++k) {
          double akp = A[IDX(k, p, n)], akq = A[IDX(k, q, n)];
          A[IDX(k, p, n)] = c * akp - s * akq;
          A[IDX(k, q, n)] = s * akp + c * akq;
        }
        /* A <- J^T A (rows p, q) */
        for (int k = 0; k < n; ++k) {
          double apk = A[IDX(p, k, n)], aqk = A[IDX(q, k, n)];
          A[IDX(p, k, n)] = c * apk - s * aqk;
          A[IDX(q, k, n)] = s * apk + c * aqk;
        }
        A[IDX(p, q, n)] = 0.0;
        A[IDX(q, p, n)] = 0.0;
        /* V <- V J */
        for (int k = 0; k < n; ++k) {
          double vkp = V[IDX(k, p, n)], vkq = V[IDX(k, q, n)];
          V[IDX(k, p, n)] = c * vkp - s * vkq;
          V[IDX(k, q, n)] = s * vkp + c * vkq;
        }
        rotated = 1;
      }
    ++sweeps;
    if (!rotated) converged = 1;
  }
  for (int i = 0; i < n; ++i) lam[i] = A[IDX(i, i, n)];
  /* selection sort ascending, moving eigenvector columns along */
  double* tmp = dalloc(n);
  for (int i = 0; i < n - 1; ++i) {
    int k = i;
    for (int j = i + 1; j < n; ++j)
      if (lam[j] < lam[k]) k = j;
    if (k != i) {
      double tl = lam[i]; lam[i] = lam[k]; lam[k] = tl;
      memcpy(tmp, &V[IDX(0, i, n)], sizeof(double) * n);
      memcpy(&V[IDX(0, i, n)], &V[IDX(0, k, n)], sizeof(double) * n);
      memcpy(&V[IDX(0, k, n)], tmp, sizeof(double) * n);
    }
  }
  free(tmp);
  free(A);
  return converged ? sweeps : -1;
}

/* Pi_{S+}(A) = sum_{lambda_i > 0} lambda_i v_i v_i^T (Eq. 2).  Optionally
 * returns the number of positive and negative eigenvalues. */
int orc_psd_project(int n, const double* A, double* out, int* npos, int* nneg) {
  double* lam = dalloc(n);
  double* V = dalloc((size_t)n * n);
  int sw = orc_jacobi_eig(n, A, lam, V);
  int np = 0, nn = 0;
  for (size_t t = 0; t < (size_t)n * n; ++t) out[t] = 0.0;
  for (int k = 0; k < n; ++k) {
    if (lam[k] > 0.0) {
      ++np;
      for (int j = 0; j < n; ++j) {
        double vj = lam[k] * V[IDX(j, k, n)];
        for (int i = 0; i < n; ++i) out[IDX(i, j, n)] += V[IDX(i, k, n)] * vj;
      }
    } else if (lam[k] < 0.0) {
      ++nn;
    }
  }
  if (npos) *npos = np;
  if (nneg) *nneg = nn;
  free(lam);
  free(V);
  return sw < 0 ? ORC_E_NUMERICAL : ORC_OK;
}

/* Dense Cholesky A = L L^T (lower, column-major).  Returns 0 on success and
 * the (1-based) index of the first non-positive pivot otherwise. */
int orc_cholesky(int n, const double* A, double* L) {
  for (size_t t = 0; t < (size_t)n * n; ++t) L[t] = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = A[IDX(j, j, n)];
    for (int k = 0; k < j; ++k) d -= L[IDX(j, k, n)] * L[IDX(j, k, n)];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    L[IDX(j, j, n)] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[IDX(i, j, n)];
      for (int k = 0; k < j; ++k) s -= L[IDX(i, k, n)] * L[IDX(j, k, n)];
      L[IDX(i, j, n)] = s / ljj;
    }
  }
  return 0;
}

/* 1 if M + shift*I is positive definite (Cholesky succeeds), else 0. */
int orc_is_pd_shifted(int n, const double* M, double shift) {
  double* A = dalloc((size_t)n * n);
  double* L = dalloc((size_t)n * n);
  memcpy(A, M, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i) A[IDX(i, i, n)] += shift;
  int r = orc_cholesky(n, A, L);
  free(A);
  free(L);
  return r == 0;
}

/* ------------------------------------------------------------------ */
/* Constraint operator.  Constraint p is the symmetric matrix A_p given */
/* by COO entries (p, i, j, v) with i <= j; an off-diagonal entry stands */
/* for both (i,j) and (j,i).  A(X)_p = <A_p, X>_F; A^T(u) = sum u_p A_p. */
/* ------------------------------------------------------------------ */
typedef struct {
  int n, m;
  long nnz;
  const int *cp, *ci, *cj;
  const double* cv;
} orc_cons;

void orc_A(const orc_cons* A, const double* X, double* u) {
  for (int p = 0; p < A->m; ++p) u[p] = 0.0;
  for (long t = 0; t < A->nnz; ++t) {
    int i = A->ci[t], j = A->cj[t];
    double w = (i == j) ? 1.0 : 2.0;
    u[A->cp[t]] += w * A->cv[t] * X[IDX(i, j, A->n)];
  }
}

/* X <- X + scale * A^T(u) */
void orc_AT_add(const orc_cons* A, const double* u, double scale, double* X) {
  for (long t = 0; t < A->nnz; ++t) {
    int i = A->ci[t], j = A->cj[t];
    double v = scale * u[A->cp[t]] * A->cv[t];
    X[IDX(i, j, A->n)] += v;
    if (i != j) X[IDX(j, i, A->n)] += v;
  }
}

/* ------------------------------------------------------------------ */
/* Linear step (Eq. kkt_system with P = 0):                            */
/*   ((sigma+rho) I + rho A^T A) x~ = r                                */
/*   x~ = (r - rho A^T K^{-1} A(r)) / s,   K = s I_m + rho A A^T.       */
/* K is eliminated by blocks: D = an independent set of constraints in */
/* the sparsity graph of A A^T (so K_DD is diagonal), F = the rest,    */
/* Schur complement S = K_FF - K_FD K_DD^{-1} K_DF factored by Cholesky.*/
/* ------------------------------------------------------------------ */
typedef struct {
  int m, nF;
  double s, rho;
  int* inD;       /* m: 1 if in D */
  int* fpos;      /* m: position in F or -1 */
  int* Flist;     /* nF */
  double* Kdiag;  /* m: K_pp */
  /* off-diagonal entries of K in CSR over rows (only (d,f) and (f,d), f,f) */
  long* rowptr;   /* m+1 */
  int* colidx;
  double* val;
  double* Lf;     /* nF x nF Cholesky factor of S */
} orc_kfac;

typedef struct { int p, q; double v; } trip;
typedef struct { int i, j; long t; } ent;

static int cmp_ent(const void* a, const void* b) {
  const ent* x = (const ent*)a; const ent* y = (const ent*)b;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return (x->t < y->t) ? -1 : (x->t > y->t);
}
static int cmp_trip(const void* a, const void* b) {
  const trip* x = (const trip*)a; const trip* y = (const trip*)b;
  if (x->p != y->p) return x->p < y->p ? -1 : 1;
  if (x->q != y->q) return x->q < y->q ? -1 : 1;
  return 0;
}

static int* g_deg_for_sort;
static int cmp_by_degree(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  if (g_deg_for_sort[x] != g_deg_for_sort[y]) return g_deg_for_sort[x] < g_deg_for_sort[y] ? -1 : 1;
  return x < y ? -1 : (x > y);
}

void orc_kfree(orc_kfac* K) {
  if (!K) return;
  free(K->inD); free(K->fpos); free(K->Flist); free(K->Kdiag);
  free(K->rowptr); free(K->colidx); free(K->val); free(K->Lf);
  free(K);
}

orc_kfac* orc_kfactor(const orc_cons* A, double sigma, double rho) {
  int m = A->m;
  double s = sigma + rho;
  orc_kfac* K = (orc_kfac*)calloc(1, sizeof(orc_kfac));
  K->m = m; K->s = s; K->rho = rho;
  /* group COO entries by matrix position (i,j) */
  ent* E = (ent*)malloc(sizeof(ent) * (A->nnz ? A->nnz : 1));
  for (long t = 0; t < A->nnz; ++t) { E[t].i = A->ci[t]; E[t].j = A->cj[t]; E[t].t = t; }
  qsort(E, A->nnz, sizeof(ent), cmp_ent);
  /* triplets of A A^T: (A A^T)_pq = sum over positions (A_p)_ij (A_q)_ij, */
  /* each off-diagonal position counted twice (i,j) and (j,i).           */
  long ntrip = 0, cap = 16;
  trip* T = (trip*)malloc(sizeof(trip) * cap);
  long g0 = 0;
  while (g0 < A->nnz) {
    long g1 = g0;
    while (g1 < A->nnz && E[g1].i == E[g0].i && E[g1].j == E[g0].j) ++g1;
    double w = (E[g0].i == E[g0].j) ? 1.0 : 2.0;
    for (long a = g0; a < g1; ++a)
      for (long b = g0; b < g1; ++b) {
        if (ntrip == cap) { cap *= 2; T = (trip*)realloc(T, sizeof(trip) * cap); }
        T[ntrip].p = A->cp[E[a].t];
        T[ntrip].q = A->cp[E[b].t];
        T[ntrip].v = w * A->cv[E[a].t] * A->cv[E[b].t];
        ++ntrip;
      }
    g0 = g1;
  }
  free(E);
  qsort(T, ntrip, sizeof(trip), cmp_trip);
  /* merge duplicates */
  long nu = 0;
  for (long t = 0; t < ntrip; ++t) {
    if (nu > 0 && T[nu - 1].p == T[t].p && T[nu - 1].q == T[t].q) T[nu - 1].v += T[t].v;
    else T[nu++] = T[t];
  }
  K->Kdiag = dalloc(m);
  for (int p = 0; p < m; ++p) K->Kdiag[p] = s;
  int* deg = (int*)calloc(m ? m : 1, sizeof(int));
  long noff = 0;
  for (long t = 0; t < nu; ++t) {
    if (T[t].p == T[t].q) K->Kdiag[T[t].p] += rho * T[t].v;
    else if (T[t].v != 0.0) { deg[T[t].p]++; ++noff; }
  }
  K->rowptr = (long*)calloc(m + 1, sizeof(long));
  K->colidx = (int*)malloc(sizeof(int) * (noff ? noff : 1));
  K->val = dalloc(noff);
  {
    long k = 0;
    for (long t = 0; t < nu; ++t) {
      if (T[t].p == T[t].q || T[t].v == 0.0) continue;
      K->colidx[k] = T[t].q;
      K->val[k] = rho * T[t].v;
      K->rowptr[T[t].p + 1]++;
      ++k;
    }
    for (int p = 0; p < m; ++p) K->rowptr[p + 1] += K->rowptr[p];
  }
  free(T);
  /* greedy independent set D, lowest degree first */
  int* order = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  for (int p = 0; p < m; ++p) order[p] = p;
  g_deg_for_sort = deg;
  qsort(order, m, sizeof(int), cmp_by_degree);
  K->inD = (int*)calloc(m ? m : 1, sizeof(int));
  for (int a = 0; a < m; ++a) {
    int p = order[a], ok = 1;
    for (long k = K->rowptr[p]; k < K->rowptr[p + 1]; ++k)
      if (K->inD[K->colidx[k]]) { ok = 0; break; }
    K->inD[p] = ok;
  }
  free(order);
  free(deg);
  K->fpos = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  K->nF = 0;
  for (int p = 0; p < m; ++p) K->fpos[p] = K->inD[p] ? -1 : K->nF++;
  K->Flist = (int*)malloc(sizeof(int) * (K->nF ? K->nF : 1));
  for (int p = 0; p < m; ++p) if (!K->inD[p]) K->Flist[K->fpos[p]] = p;
  /* Schur complement S = K_FF - K_FD K_DD^{-1} K_DF */
  int nF = K->nF;
  double* S = dalloc((size_t)nF * nF);
  for (int a = 0; a < nF; ++a) {
    int p = K->Flist[a];
    S[IDX(a, a, nF)] = K->Kdiag[p];
    for (long k = K->rowptr[p]; k < K->rowptr[p + 1]; ++k) {
      int q = K->colidx[k];
      if (!K->inD[q]) S[IDX(a, K->fpos[q], nF)] += K->val[k];
    }
  }
  for (int d = 0; d < m; ++d) {
    if (!K->inD[d]) continue;
    for (long k1 = K->rowptr[d]; k1 < K->rowptr[d + 1]; ++k1)
      for (long k2 = K->rowptr[d]; k2 < K->rowptr[d + 1]; ++k2) {
        int a = K->fpos[K->colidx[k1]], b = K->fpos[K->colidx[k2]];
        S[IDX(a, b, nF)] -= K->val[k1] * K->val[k2] / K->Kdiag[d];
      }
  }
  K->Lf = dalloc((size_t)nF * nF);
  int bad = orc_cholesky(nF, S, K->Lf);
  free(S);
  if (bad) { orc_kfree(K); return NULL; }
  return K;
}

/* v = K^{-1} u */
void orc_ksolve(const orc_kfac* K, const double* u, double* v) {
  int m = K->m, nF = K->nF;
  double* t = dalloc(nF);
  for (int a = 0; a < nF; ++a) {
    int f = K->Flist[a];
    double acc = u[f];
    for (long k = K->rowptr[f]; k < K->rowptr[f + 1]; ++k) {
      int d = K->colidx[k];
      if (K->inD[d]) acc -= K->val[k] * u[d] / K->Kdiag[d];
    }
    t[a] = acc;
  }
  /* S vF = t : forward then backward substitution with Lf */
  for (int i = 0; i < nF; ++i) {
    double acc = t[i];
    for (int k = 0; k < i; ++k) acc -= K->Lf[IDX(i, k, nF)] * t[k];
    t[i] = acc / K->Lf[IDX(i, i, nF)];
  }
  for (int i = nF - 1; i >= 0; --i) {
    double acc = t[i];
    for (int k = i + 1; k < nF; ++k) acc -= K->Lf[IDX(k, i, nF)] * t[k];
    t[i] = acc / K->Lf[IDX(i, i, nF)];
  }
  for (int a = 0; a < nF; ++a) v[K->Flist[a]] = t[a];
  for (int d = 0; d < m; ++d) {
    if (!K->inD[d]) continue;
    double acc = u[d];
    for (long k = K->rowptr[d]; k < K->rowptr[d + 1]; ++k) {
      int f = K->colidx[k];
      if (!K->inD[f]) acc -= K->val[k] * v[f];
    }
    v[d] = acc / K->Kdiag[d];
  }
  free(t);
}

int orc_kfactor_nF(const orc_kfac* K) { return K ? K->nF : -1; }

/* x~ = ((sigma+rho) I + rho A^T A)^{-1} r  (standalone, for tests) */
int orc_linear_step(const orc_cons* A, double sigma, double rho, const double* r, double* xt) {
  orc_kfac* K = orc_kfactor(A, sigma, rho);
  if (!K) return ORC_E_NUMERICAL;
  int n = A->n, m = A->m;
  double* u = dalloc(m);
  double* v = dalloc(m);
  orc_A(A, r, u);
  orc_ksolve(K, u, v);
  for (size_t t = 0; t < (size_t)n * n; ++t) xt[t] = r[t];
  orc_AT_add(A, v, -rho, xt);
  for (size_t t = 0; t < (size_t)n * n; ++t) xt[t] /= K->s;
  free(u); free(v);
  orc_kfree(K);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: Rayleigh-Ritz on span(S), S n x p.  Orthonormalise S by */
/* Cholesky QR (Q = S L^{-T}, L = chol(S^T S)), eigendecompose Q^T A Q  */
/* ascending, return Ritz vectors Q W~ (n x p) and values (p).         */
/* Returns 0, or ORC_E_NUMERICAL when the Cholesky QR breaks down.     */
/* ------------------------------------------------------------------ */
int orc_rayleigh_ritz(int n, const double* A, int p, const double* S, double* ritz_vec, double* ritz_val) {
  if (p == 0) return ORC_OK;
  double* G = dalloc((size_t)p * p);
  double* L = dalloc((size_t)p * p);
  gemm_tn(n, p, p, S, S, G);
  int bad = orc_cholesky(p, G, L);
  if (bad) { free(G); free(L); return ORC_E_NUMERICAL; }
  /* Q = S L^{-T}: row-wise forward substitution  Q L^T = S */
  double* Q = dalloc((size_t)n * p);
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < p; ++j) {
      double acc = S[IDX(r, j, n)];
      for (int k = 0; k < j; ++k) acc -= Q[IDX(r, k, n)] * L[IDX(j, k, p)];
      Q[IDX(r, j, n)] = acc / L[IDX(j, j, p)];
    }
  double* AQ = dalloc((size_t)n * p);
  gemm_nn(n, n, p, A, Q, AQ);
  double* H = dalloc((size_t)p * p);
  gemm_tn(n, p, p, Q, AQ, H);
  double* U = dalloc((size_t)p * p);
  int sw = orc_jacobi_eig(p, H, ritz_val, U);
  gemm_nn(n, p, p, Q, U, ritz_vec);
  free(G); free(L); free(Q); free(AQ); free(H); free(U);
  return sw < 0 ? ORC_E_NUMERICAL : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3: LOBPCG for the positive eigenpairs of symmetric A.     */
/*  X (n x mcap) holds X^0 in its first *m_io columns on entry and the */
/*  Ritz vectors on exit; lam (mcap) the Ritz values (ascending).      */
/*  Stops when every Ritz pair of the block has ||A x - theta x||_2 <= */
/*  tol (Section 5), no column being a fresh random one; checked       */
/*  before each Rayleigh-Ritz step.  Gives up after maxit RR steps.    */
/*  Expansion: if more than m Ritz values of the trial subspace are    */
/*  positive, X^{k+1} = [m largest Ritz vectors, b Gaussian columns];  */
/*  the Gaussian columns enter the next trial subspace with their      */
/*  residual A g (any Ritz value gives the same span), and Delta X     */
/*  keeps only the columns that have a predecessor.                    */
/*  Columns of R and Delta X are scaled to unit norm before Cholesky   */
/*  QR (this leaves the trial subspace unchanged).  On a Cholesky QR   */
/*  breakdown the step is retried without Delta X.                     */
/* info[0] = RR steps, info[1] = expansions, info[2] = 1 if converged, */
/* info[3] = number of positive Ritz values at exit.                   */
/* resn (mcap) receives the final residual norms.                      */
/* Returns ORC_OK, ORC_E_NUMERICAL (breakdown) or ORC_E_NOMEM when the */
/* block would exceed mcap columns.                                    */
/* ------------------------------------------------------------------ */
int orc_lobpcg(int n, const double* A, int* m_io, int mcap, double* X, double* lam, double tol, int maxit,
               int bexp, uint64_t seed, uint32_t stream, int* info, double* resn) {
  int m = *m_io;
  if (m <= 0 || m > mcap || m > n) return ORC_E_INVALID;
  size_t nm = (size_t)n * mcap;
  double* Sbuf = dalloc((size_t)n * 3 * mcap);
  double* RV = dalloc((size_t)n * 3 * mcap);
  double* RL = dalloc(3 * mcap);
  double* AX = dalloc(nm);
  double* R = dalloc(nm);
  double* DX = dalloc(nm);
  double* Xold = dalloc(nm);
  int mdx = 0;        /* columns in Delta X */
  int nfresh = 0;     /* trailing Gaussian columns not yet Ritz vectors */
  int status = ORC_OK;
  info[0] = info[1] = info[2] = info[3] = 0;
  /* initial Rayleigh-Ritz on span(X^0) (Algorithm 3) */
  if (orc_rayleigh_ritz(n, A, m, X, RV, RL)) { status = ORC_E_NUMERICAL; goto done; }
  memcpy(X, RV, sizeof(double) * (size_t)n * m);
  memcpy(lam, RL, sizeof(double) * m);
  for (int it = 0;; ++it) {
    /* R = A X - X Lambda (fresh columns: Lambda = 0) */
    gemm_nn(n, n, m, A, X, AX);
    int allconv = (nfresh == 0), npos = 0;
    for (int j = 0; j < m; ++j) {
      double th = (j < m - nfresh) ? lam[j] : 0.0;
      double nr = 0.0;
      for (int i = 0; i < n; ++i) {
        double r = AX[IDX(i, j, n)] - th * X[IDX(i, j, n)];
        R[IDX(i, j, n)] = r;
        nr += r * r;
      }
      nr = sqrt(nr);
      resn[j] = nr;
      if (j < m - nfresh && th > 0.0) ++npos;
      if (nr > tol) allconv = 0;
    }
    info[3] = npos;
    if (allconv) { info[2] = 1; break; }
    if (it >= maxit) break;
    /* Rayleigh-Ritz on span(X, R, Delta X), keep the m largest (Algorithm 3) */
    int use_dx = (mdx > 0);
    int rc = 1;
    int p = 0;
    for (int attempt = 0; attempt < 2 && rc; ++attempt) {
      p = 0;
      memcpy(Sbuf, X, sizeof(double) * (size_t)n * m);
      p += m;
      for (int j = 0; j < m; ++j) {
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += R[IDX(i, j, n)] * R[IDX(i, j, n)];
        nr = sqrt(nr);
        if (nr == 0.0) continue; /* a zero residual adds nothing to the span */
        for (int i = 0; i < n; ++i) Sbuf[IDX(i, p, n)] = R[IDX(i, j, n)] / nr;
        ++p;
      }
      if (use_dx)
        for (int j = 0; j < mdx; ++j) {
          double nr = 0.0;
          for (int i = 0; i < n; ++i) nr += DX[IDX(i, j, n)] * DX[IDX(i, j, n)];
          nr = sqrt(nr);
          if (nr == 0.0) continue;
          for (int i = 0; i < n; ++i) Sbuf[IDX(i, p, n)] = DX[IDX(i, j, n)] / nr;
          ++p;
        }
      if (p > n) p = n; /* cannot exceed the dimension; keep the leading columns */
      rc = orc_rayleigh_ritz(n, A, p, Sbuf, RV, RL);
      if (rc) use_dx = 0;
    }
    if (rc) { status = ORC_E_NUMERICAL; break; }
    info[0]++;
    int npos_rr = 0;
    for (int j = 0; j < p; ++j) if (RL[j] > 0.0) ++npos_rr;
    int mkeep = m < p ? m : p;
    /* Delta X^{k+1} = X^{k+1} - X^k; sign of each new Ritz vector aligned */
    /* with its predecessor column (eigenvectors are defined up to sign).  */
    memcpy(Xold, X, sizeof(double) * (size_t)n * m);
    for (int j = 0; j < mkeep; ++j) {
      int src = p - mkeep + j;
      lam[j] = RL[src];
      double dot = 0.0;
      for (int i = 0; i < n; ++i) dot += RV[IDX(i, src, n)] * Xold[IDX(i, j, n)];
      double sg = (dot < 0.0) ? -1.0 : 1.0;
      for (int i = 0; i < n; ++i) X[IDX(i, j, n)] = sg * RV[IDX(i, src, n)];
    }
    mdx = 0;
    for (int j = 0; j < mkeep && j < m - nfresh; ++j) {
      for (int i = 0; i < n; ++i) DX[IDX(i, mdx, n)] = X[IDX(i, j, n)] - Xold[IDX(i, j, n)];
      ++mdx;
    }
    nfresh = 0;
    m = mkeep;
    /* expansion of the block (Algorithm 3) */
    if (npos_rr > m) {
      int b = bexp;
      if (m + b > mcap || m + b > n) { status = ORC_E_NOMEM; break; }
      for (int j = 0; j < b; ++j)
        for (int i = 0; i < n; ++i)
          X[IDX(i, m + j, n)] = orc_normal(seed, stream, (uint32_t)info[1], (uint32_t)i, (uint32_t)j);
      for (int j = 0; j < b; ++j) lam[m + j] = 0.0;
      m += b;
      nfresh = b;
      info[1]++;
    }
  }
done:
  *m_io = m;
  free(Sbuf); free(RV); free(RL); free(AX); free(R); free(DX); free(Xold);
  (void)nm;
  return status;
}

/* Standalone projection by LOBPCG (Algorithm 3 for the positive
 * eigenpairs from the warm block X, n x *m_io of an n x mcap buffer) and
 * the reconstruction Pi(A) = sum over positive Ritz values theta x x^T
 * (Eq. 2, first form).  out: n x n.  Returns the LOBPCG status. */
int orc_lobpcg_project(int n, const double* A, int* m_io, int mcap, double* X, double tol, int maxit, double* out,
                       int* info) {
  double* lam = dalloc(mcap);
  double* resn = dalloc(mcap);
  int bexp = (int)ceil(n / 50.0);
  if (bexp < 1) bexp = 1;
  int rc = orc_lobpcg(n, A, m_io, mcap, X, lam, tol, maxit, bexp, 0, 0, info, resn);
  for (size_t t = 0; t < (size_t)n * n; ++t) out[t] = 0.0;
  if (rc == ORC_OK) {
    for (int k = 0; k < *m_io; ++k) {
      if (!(lam[k] > 0.0)) continue;
      for (int j = 0; j < n; ++j) {
        double vj = lam[k] * X[IDX(j, k, n)];
        for (int i = 0; i < n; ++i) out[IDX(i, j, n)] += X[IDX(i, k, n)] * vj;
      }
    }
  }
  free(lam);
  free(resn);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 on min <C,X> s.t. A(X) = b, X psd.                      */
/* ------------------------------------------------------------------ */
typedef struct {
  double rho, sigma, alpha;
  double eps_abs, eps_rel, eps_pinf, eps_dinf;
  int max_iter, check_every;
  int use_lobpcg;          /* 0: exact projection every iteration */
  int lobpcg_maxit;        /* cap on Rayleigh-Ritz steps per projection */
  double tol_coef, tol_exp;/* LOBPCG tolerance tol_coef / k^tol_exp */
  double expand_frac;      /* b = ceil(expand_frac * n) */
  double mode_frac;        /* 1/3 */
  uint64_t seed;
} orc_settings;

typedef struct {
  int status, iters;
  double obj, r_prim, r_dual;
  int n_exact, n_lobpcg, lobpcg_steps, expansions, last_rank;
  int n_neg;               /* LOBPCG projections done in negative mode (on -W) */
} orc_info;

#define MODE_POS 0
#define MODE_NEG 1
#define MODE_EXACT 2

static double maxabs(const double* a, size_t k) {
  double r = 0.0;
  for (size_t t = 0; t < k; ++t) if (fabs(a[t]) > r) r = fabs(a[t]);
  return r;
}

/* Seed an LOBPCG block from a full eigendecomposition (lam ascending). */
static int seed_block(int n, int mode, const double* lam, const double* V, int count, int b, int mcap, double* X) {
  int m = count + b;
  if (m > mcap) m = mcap;
  if (m > n) m = n;
  if (m < 1) m = 1;
  for (int j = 0; j < m; ++j) {
    int src = (mode == MODE_POS) ? (n - 1 - j) : j; /* largest of W, or largest of -W */
    memcpy(&X[IDX(0, j, n)], &V[IDX(0, src, n)], sizeof(double) * n);
  }
  return m;
}

/*
 * Inputs: n, C (n x n), constraints A (m, COO), b (m).
 * Outputs (caller-allocated): x, Z, Y (n x n), ye (m), cert (n*n + m):
 *   PRIMAL_INFEASIBLE -> cert = [y-bar_e (m); Y-bar (n*n)]
 *   DUAL_INFEASIBLE   -> cert = [0 (m); x-bar (n*n)]
 */
int orc_admm_solve(int n, const double* C, const orc_cons* A, const double* b, const orc_settings* st,
                   double* x, double* Z, double* Y, double* ye, double* cert, orc_info* info) {
  int m = A->m;
  size_t nn = (size_t)n * n;
  double rho = st->rho, sigma = st->sigma, alpha = st->alpha, s = sigma + rho;
  memset(info, 0, sizeof(*info));
  orc_kfac* K = orc_kfactor(A, sigma, rho);
  if (!K) return ORC_E_NUMERICAL;
  double *ze = dalloc(m), *t = dalloc(m), *u = dalloc(m), *v = dalloc(m), *zt = dalloc(m), *we = dalloc(m);
  double *r = dalloc(nn), *xt = dalloc(nn), *W = dalloc(nn), *Wneg = dalloc(nn);
  double *xprev = dalloc(nn), *Yprev = dalloc(nn), *yeprev = dalloc(m);
  double *lam = dalloc(n), *V = dalloc(nn), *tmp = dalloc(nn), *tmpm = dalloc(m);
  int bexp = (int)ceil(st->expand_frac * n);
  if (bexp < 1) bexp = 1;
  int mcap = (int)ceil(st->mode_frac * n) + bexp;
  if (mcap > n) mcap = n;
  double* Xb = dalloc((size_t)n * mcap);
  double* th = dalloc(mcap);
  double* resn = dalloc(mcap);
  int mode = MODE_EXACT, mblk = 0;
  int status = ORC_MAX_ITER;
  for (size_t q = 0; q < nn; ++q) x[q] = Z[q] = Y[q] = 0.0;
  for (int p = 0; p < m; ++p) ye[p] = ze[p] = 0.0;
  int k;
  for (k = 1; k <= st->max_iter; ++k) {
    int check = (k % st->check_every) == 0;
    if (check) {
      memcpy(xprev, x, sizeof(double) * nn);
      memcpy(Yprev, Y, sizeof(double) * nn);
      memcpy(yeprev, ye, sizeof(double) * m);
    }
    /* linear step (Algorithm 1).  r = sigma x - q + rho A-bar^T (z - y/rho) */
    for (int p = 0; p < m; ++p) t[p] = ze[p] - ye[p] / rho;
    for (size_t q = 0; q < nn; ++q) r[q] = sigma * x[q] - C[q] + rho * (Z[q] - Y[q] / rho);
    orc_AT_add(A, t, rho, r);
    orc_A(A, r, u);
    orc_ksolve(K, u, v);
    for (size_t q = 0; q < nn; ++q) xt[q] = r[q];
    orc_AT_add(A, v, -rho, xt);
    for (size_t q = 0; q < nn; ++q) xt[q] /= s;
    orc_A(A, xt, zt); /* z~ = A-bar x~ : equality block A(x~), cone block x~ */
    /* relaxed primal update (Algorithm 1): x <- alpha x~ + (1-alpha) x */
    for (size_t q = 0; q < nn; ++q) x[q] = alpha * xt[q] + (1.0 - alpha) * x[q];
    /* projection step (Algorithm 1): z <- Pi_C(alpha z~ + (1-alpha) z + y/rho) */
    for (int p = 0; p < m; ++p) we[p] = alpha * zt[p] + (1.0 - alpha) * ze[p] + ye[p] / rho;
    for (size_t q = 0; q < nn; ++q) W[q] = alpha * xt[q] + (1.0 - alpha) * Z[q] + Y[q] / rho;
    /* projection onto S+ */
    int done_proj = 0;
    if (st->use_lobpcg && k > 1 && mode != MODE_EXACT) {
      const double* Aproj = W;
      if (mode == MODE_NEG) {
        for (size_t q = 0; q < nn; ++q) Wneg[q] = -W[q];
        Aproj = Wneg;
      }
      double tol = st->tol_coef / pow((double)k, st->tol_exp);
      int li[4];
      int mm = mblk;
      int rc = orc_lobpcg(n, Aproj, &mm, mcap, Xb, th, tol, st->lobpcg_maxit, bexp, st->seed, (uint32_t)k, li, resn);
      if (rc == ORC_OK) {
        mblk = mm;
        info->n_lobpcg++;
        if (mode == MODE_NEG) info->n_neg++;
        info->lobpcg_steps += li[0];
        info->expansions += li[1];
        /* reconstruction: POS Z = sum theta x x^T ; NEG Z = W + sum theta x x^T */
        if (mode == MODE_POS) for (size_t q = 0; q < nn; ++q) Z[q] = 0.0;
        else memcpy(Z, W, sizeof(double) * nn);
        int npos = 0;
        for (int j = 0; j < mblk; ++j) {
          if (!(th[j] > 0.0)) continue;
          ++npos;
          for (int c = 0; c < n; ++c) {
            double vc = th[j] * Xb[IDX(c, j, n)];
            for (int i = 0; i < n; ++i) Z[IDX(i, c, n)] += Xb[IDX(i, j, n)] * vc;
          }
        }
        info->last_rank = npos;
        /* next mode from the counts (Section 5) */
        int cnt_pos = (mode == MODE_POS) ? npos : n - npos;
        int cnt_neg = (mode == MODE_POS) ? n - npos : npos;
        int next = (cnt_pos < st->mode_frac * n) ? MODE_POS : (cnt_neg < st->mode_frac * n) ? MODE_NEG : MODE_EXACT;
        if (next != mode) { mode = MODE_EXACT; } /* re-seed through an exact step */
        done_proj = 1;
      }
    }
    if (!done_proj) {
      int sw = orc_jacobi_eig(n, W, lam, V);
      if (sw < 0) { status = ORC_E_NUMERICAL; break; }
      for (size_t q = 0; q < nn; ++q) Z[q] = 0.0;
      int npos = 0, nneg = 0;
      for (int j = 0; j < n; ++j) {
        if (lam[j] > 0.0) {
          ++npos;
          for (int c = 0; c < n; ++c) {
            double vc = lam[j] * V[IDX(c, j, n)];
            for (int i = 0; i < n; ++i) Z[IDX(i, c, n)] += V[IDX(i, j, n)] * vc;
          }
        } else if (lam[j] < 0.0) {
          ++nneg;
        }
      }
      info->n_exact++;
      info->last_rank = npos;
      if (st->use_lobpcg) {
        if (npos < st->mode_frac * n) {
          mode = MODE_POS;
          mblk = seed_block(n, MODE_POS, lam, V, npos, bexp, mcap, Xb);
        } else if (nneg < st->mode_frac * n) {
          mode = MODE_NEG;
          mblk = seed_block(n, MODE_NEG, lam, V, nneg, bexp, mcap, Xb);
        } else {
          mode = MODE_EXACT;
        }
      }
    }
    for (int p = 0; p < m; ++p) ze[p] = b[p];
    /* dual update (Algorithm 1): y <- y + rho (alpha z~ + (1-alpha) z - z+) */
    for (int p = 0; p < m; ++p) ye[p] = rho * (we[p] - b[p]);
    for (size_t q = 0; q < nn; ++q) Y[q] = rho * (W[q] - Z[q]);
    if (!check) continue;
    /* termination (Section 5 footnote: checked every check_every iterations) */
    orc_A(A, x, tmpm);
    double rp = 0.0, nAx = 0.0, nz = maxabs(ze, m);
    for (int p = 0; p < m; ++p) {
      if (fabs(tmpm[p] - ze[p]) > rp) rp = fabs(tmpm[p] - ze[p]);
      if (fabs(tmpm[p]) > nAx) nAx = fabs(tmpm[p]);
    }
    for (size_t q = 0; q < nn; ++q) {
      if (fabs(x[q] - Z[q]) > rp) rp = fabs(x[q] - Z[q]);
      if (fabs(x[q]) > nAx) nAx = fabs(x[q]);
      if (fabs(Z[q]) > nz) nz = fabs(Z[q]);
    }
    for (size_t q = 0; q < nn; ++q) tmp[q] = Y[q];
    orc_AT_add(A, ye, 1.0, tmp); /* A-bar^T y */
    double rd = 0.0, nATy = maxabs(tmp, nn), nC = maxabs(C, nn);
    for (size_t q = 0; q < nn; ++q) if (fabs(C[q] + tmp[q]) > rd) rd = fabs(C[q] + tmp[q]);
    double obj = 0.0;
    for (size_t q = 0; q < nn; ++q) obj += C[q] * x[q];
    info->obj = obj; info->r_prim = rp; info->r_dual = rd; info->iters = k;
    double ep = st->eps_abs + st->eps_rel * (nAx > nz ? nAx : nz);
    double ed = st->eps_abs + st->eps_rel * (nC > nATy ? nC : nATy);
    if (rp <= ep && rd <= ed) { status = ORC_SOLVED; break; }
    /* primal infeasibility: delta y = y^k - y^{k-1} */
    double ndy = 0.0;
    for (int p = 0; p < m; ++p) if (fabs(ye[p] - yeprev[p]) > ndy) ndy = fabs(ye[p] - yeprev[p]);
    for (size_t q = 0; q < nn; ++q) if (fabs(Y[q] - Yprev[q]) > ndy) ndy = fabs(Y[q] - Yprev[q]);
    if (ndy > 1e-12) {
      for (int p = 0; p < m; ++p) tmpm[p] = (ye[p] - yeprev[p]) / ndy;     /* y-bar_e */
      for (size_t q = 0; q < nn; ++q) tmp[q] = (Y[q] - Yprev[q]) / ndy;   /* Y-bar  */
      double bty = 0.0;
      for (int p = 0; p < m; ++p) bty += b[p] * tmpm[p];
      for (size_t q = 0; q < nn; ++q) r[q] = tmp[q];
      orc_AT_add(A, tmpm, 1.0, r); /* A-bar^T y-bar */
      double nat = maxabs(r, nn);
      if (nat < st->eps_pinf && bty < -st->eps_pinf) {
        for (size_t q = 0; q < nn; ++q) r[q] = -tmp[q];
        if (orc_is_pd_shifted(n, r, st->eps_pinf)) {
          memcpy(cert, tmpm, sizeof(double) * m);
          memcpy(cert + m, tmp, sizeof(double) * nn);
          status = ORC_PRIMAL_INFEASIBLE;
          break;
        }
      }
    }
    /* dual infeasibility: delta x = x^k - x^{k-1} */
    double ndx = 0.0;
    for (size_t q = 0; q < nn; ++q) if (fabs(x[q] - xprev[q]) > ndx) ndx = fabs(x[q] - xprev[q]);
    if (ndx > 1e-12) {
      for (size_t q = 0; q < nn; ++q) tmp[q] = (x[q] - xprev[q]) / ndx;
      orc_A(A, tmp, tmpm);
      double nax = maxabs(tmpm, m);
      double ctx = 0.0;
      for (size_t q = 0; q < nn; ++q) ctx += C[q] * tmp[q];
      if (nax < st->eps_dinf && ctx < -st->eps_dinf && orc_is_pd_shifted(n, tmp, st->eps_dinf)) {
        for (int p = 0; p < m; ++p) cert[p] = 0.0;
        memcpy(cert + m, tmp, sizeof(double) * nn);
        status = ORC_DUAL_INFEASIBLE;
        break;
      }
    }
  }
  if (k > st->max_iter) info->iters = st->max_iter;
  info->status = status;
  orc_kfree(K);
  free(ze); free(t); free(u); free(v); free(zt); free(we);
  free(r); free(xt); free(W); free(Wneg); free(xprev); free(Yprev); free(yeprev);
  free(lam); free(V); free(tmp); free(tmpm); free(Xb); free(th); free(resn);
  return status;
}
