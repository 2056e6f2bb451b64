/*
 * sdpgpu.h -- C ABI of the GB300 (sm_103a) approximate-ADMM SDP solver.
 *
 * Method: Rontsis, Goulart, Nakatsukasa, "Efficient Semidefinite
 * Programming with approximate ADMM".  The solver runs Algorithm 1 (ADMM)
 * on
 *
 *      minimise  <C, X>   subject to   <A_p, X> = b_p  (p = 0..m-1),  X psd,
 *
 * the dual-form SDPLIB problem of Section 5.1 written as a minimisation and
 * cast in the paper's form (P) with P = 0, q = C, A-bar = [A; I] and cone
 * {b} x S+ (Section 2).  Its projection onto the PSD cone (Eqs. 1-2) is
 * computed by a warm-started LOBPCG for the positive (or negative)
 * eigenpairs (Algorithm 3, with Rayleigh-Ritz of Algorithm 2), choosing
 * positive/negative/exact mode by the rank rule of Section 5.
 *
 * Conventions for every call:
 *  - every call returns an int status (sdp_status); negative values are
 *    errors and leave the context valid and destroyable;
 *  - matrices are dense, column-major, leading dimension n, FP64;
 *  - a pointer argument is host memory unless the call's `*_on_device` /
 *    `to_device` flag says it is device memory of the current CUDA device;
 *  - inputs are copied; the caller keeps ownership of every buffer it
 *    passes; device pointers are used only for the duration of the call;
 *  - no call keeps a pointer to caller memory after it returns;
 *  - calls on one context are not thread-safe; distinct contexts are
 *    independent.
 */
#ifndef SDPGPU_H
#define SDPGPU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdp_ctx sdp_ctx;       /* one SDP instance and its device state */
typedef struct sdp_server sdp_server; /* continuous-batching request loop     */

typedef enum {
  SDP_OK = 0,
  SDP_SOLVED = 1,             /* residuals below tolerance (Algorithm 1 converged)      */
  SDP_PRIMAL_INFEASIBLE = 2,  /* Theorem 1 (i): certificate delta-y available          */
  SDP_DUAL_INFEASIBLE = 3,    /* Theorem 1 (ii): certificate delta-x available         */
  SDP_MAX_ITER = 4,           /* iteration limit reached                               */
  SDP_RUNNING = 5,            /* (server) request admitted, not finished               */
  SDP_QUEUED = 6,             /* (server) request waiting for admission                */
  SDP_E_INVALID = -1,         /* bad argument; nothing changed                          */
  SDP_E_NOMEM = -2,           /* device allocation failed or budget exceeded            */
  SDP_E_CUDA = -3,            /* a CUDA runtime call failed                             */
  SDP_E_NUMERICAL = -4,       /* NaN/Inf or a factorisation broke down                  */
  SDP_E_TIMEOUT = -5,         /* a bounded device wait gave up                          */
  SDP_E_STATE = -6            /* call not valid in the context's current state          */
} sdp_status;

/* Precision of the projection's dense products (Section 4 block products
 * and the rank-k reconstruction of Eq. 2).  ADMM state, residuals and
 * infeasibility tests are FP64 in every mode. */
typedef enum {
  SDP_PREC_FP64 = 0,    /* every product, Gram and Rayleigh-Ritz in FP64 (CUDA cores)          */
  SDP_PREC_BF16X3 = 1,  /* W*S on tcgen05 tensor cores with split-BF16 x3, FP32 accumulate, raised to  */
                        /* the FP64-accurate split product (see sdp_dense_product) for a projection    */
                        /* whose tolerance or smallest |Ritz value| nears the x3 product's error       */
                        /* (precision ladder); block update and reconstruction in FP32 (the update     */
                        /* FP64-accurate on the tensor cores for wide blocks); Rayleigh-Ritz with its  */
                        /* Grams and Cholesky-QR FP64-accurate (FP32 by the rr_fp32 setting);          */
                        /* residual norms, ADMM state and tests FP64                                   */
  SDP_PREC_AUTO = 2     /* accepted; computes as SDP_PREC_BF16X3 (no tolerance-driven switch yet) */
} sdp_precision;

typedef struct {
  double rho;          /* ADMM step rho > 0 (Algorithm 1)                  default 1.0   */
  double sigma;        /* ADMM sigma > 0 (Algorithm 1)                     default 1e-6  */
  double alpha;        /* relaxation alpha in (0,2) (Algorithm 1)          default 1.6   */
  double eps_abs;      /* stop when r_prim, r_dual <= eps_abs + eps_rel*scale  default 1e-4 */
  double eps_rel;      /*                                                  default 0     */
  double eps_pinf;     /* primal infeasibility tolerance (Section 5.2)    default 1e-4  */
  double eps_dinf;     /* dual infeasibility tolerance (Section 5.2)      default 1e-4  */
  int max_iter;        /* ADMM iteration limit                             default 5000  */
  int check_every;     /* termination checked every this many iterations   default 40    */
  int lobpcg_max_iter; /* Rayleigh-Ritz steps per projection              default 20    */
  int precision;       /* sdp_precision                                    default FP64  */
  int exact_only;      /* 1: exact projection every iteration (comparator) default 0     */
  double tol_coef;     /* LOBPCG tolerance tol_coef / k^tol_exp (Section 5) default 10    */
  double tol_exp;      /*                                                   default 1.01  */
  double expand_frac;  /* expansion block b = ceil(expand_frac*n) (Section 4) default 1/50 */
  double mode_frac;    /* positive/negative mode threshold (Section 5)     default 1/3   */
  unsigned long long seed; /* Philox key for the random expansion columns  default 0     */
  int rr_method;       /* Rayleigh-Ritz eigensolver: 0 tridiagonal reduction (Householder,*/
                       /* Sturm bisection, inverse iteration) on one CTA while the p x p  */
                       /* matrix fits its shared memory, across the GPU above; 1 cyclic    */
                       /* Jacobi at every width (comparator)              default 0     */
  int rr_fp32;         /* 1: with BF16X3, Rayleigh-Ritz (Grams, Cholesky-QR, eigensolver)  */
                       /* in FP32 instead of FP64 -- only for spectra whose kept           */
                       /* eigenvalues are not small against ||W|| (e.g. a standalone       */
                       /* projection with a gap at zero); ADMM near a rank change needs    */
                       /* FP64                                               default 0     */
  int proj_neg;        /* sdp_project_psd only: 0 positive mode (V_warm approximates the  */
                       /* eigenvectors of the positive eigenvalues of W); 1 negative mode  */
                       /* (Section 5: V_warm approximates those of the negative ones;     */
                       /* LOBPCG runs on -W and Pi(W) = W + Pi(-W))          default 0     */
  int exact_solver;    /* eigensolver of the exact branch (Section 1's full                */
                       /* eigendecomposition; with exact_only = 1 the exact-eig ADMM       */
                       /* comparator): 0 the library's parallel cyclic Jacobi, 1 the      */
                       /* cuSOLVER syevd library routine (a comparator, not the hot path)  */
                       /*                                                    default 0     */
  int soft_lock;       /* 0: every residual and Delta X column enters the trial subspace  */
                       /* span(X, R, Delta X) of each step, as in Algorithm 3; 1: columns  */
                       /* whose residual is already within tol are left out (soft locking:*/
                       /* a narrower Rayleigh-Ritz step, but the converged pairs are not  */
                       /* improved further)                                  default 0     */
} sdp_settings;

typedef struct {
  int status;          /* final sdp_status of the solve                   */
  int iters;           /* ADMM iterations performed                        */
  double obj;          /* <C, X>                                           */
  double r_prim;       /* max(||A(X) - b||_inf, ||X - Z||_inf)             */
  double r_dual;       /* ||C + A^T(y) + Y||_inf                           */
  int n_exact;         /* projections done by full eigendecomposition      */
  int n_lobpcg;        /* projections done by LOBPCG                       */
  int lobpcg_steps;    /* Rayleigh-Ritz steps summed over projections      */
  int expansions;      /* random block expansions (Algorithm 3)            */
  int rank;            /* positive Ritz values at the last projection      */
  double solve_ms;     /* wall time of the solve (host clock)              */
  int n_neg;           /* LOBPCG projections done in negative mode         */
  int n_ladder;        /* mixed precision: LOBPCG projections whose block  */
                       /* products ran FP64-accurate (precision ladder)     */
} sdp_info;

typedef struct {
  int status;          /* SDP_OK or an error                               */
  int steps;           /* Rayleigh-Ritz steps                              */
  int m;               /* final block width                                */
  int npos;            /* positive Ritz values                             */
  int expansions;
  int converged;       /* 1 if every Ritz residual met tol                 */
  double res_fro;      /* ||R_+||_F over the positive Ritz pairs: Thm 3 gives */
                       /* ||Pi~ - Pi||_F <= sqrt(2)*res_fro (+ the perp term) */
  int jacobi_sweeps;   /* Jacobi sweeps summed over the Rayleigh-Ritz steps  */
  int mode;            /* 0 positive, 1 negative mode; 2 the exact fallback  */
                       /* (Cholesky-QR breakdown or block capacity)           */
  int fp64_products;   /* mixed precision: 1 if the block products ran       */
                       /* FP64-accurate (precision ladder), 0 split-BF16 x3   */
} sdp_proj_info;

/* Fill *s with the defaults listed above. */
void sdp_default_settings(sdp_settings* s);

/* Printable name of a status code (static storage). */
const char* sdp_status_str(int status);

/* Create a context bound to the current CUDA device.  `cuda_stream` is a
 * cudaStream_t borrowed for every later call on this context (NULL = the
 * legacy default stream).  `settings` may be NULL for the defaults.
 * Errors: SDP_E_INVALID (bad settings), SDP_E_CUDA. */
int sdp_create(sdp_ctx** ctx, const sdp_settings* settings, void* cuda_stream);

/* Load an instance (Section 5.1, Eq. sdplib as a minimisation):
 *   C     n*n column-major symmetric cost matrix;
 *   m     number of equality constraints;
 *   nnz   number of COO entries; entry t belongs to constraint p[t] and
 *         holds the value v[t] at (i[t], j[t]) with 0 <= i <= j < n; an
 *         off-diagonal entry stands for both (i,j) and (j,i), so
 *         <A_p, X> = sum over entries v * (i==j ? X_ii : 2 X_ij);
 *   b     m right-hand sides.
 * All arrays are host memory, or device memory when inputs_on_device != 0
 * (then p, i, j, v are still read once and copied).  Builds the sparse
 * operators and factors K = (sigma+rho) I_m + rho A A^T once (Algorithm 1,
 * linear step).  Errors: SDP_E_INVALID (indices out of range, n < 1),
 * SDP_E_NUMERICAL (K not positive definite), SDP_E_NOMEM. */
int sdp_setup(sdp_ctx* ctx, int n, const double* C, int m, long nnz, const int* p, const int* i,
              const int* j, const double* v, const double* b, int inputs_on_device);

/* Replace the settings of a set-up context (before sdp_solve). */
int sdp_update_settings(sdp_ctx* ctx, const sdp_settings* settings);

/* Run Algorithm 1 from the zero initial point to termination.  Returns the
 * final status (SDP_SOLVED, SDP_PRIMAL_INFEASIBLE, SDP_DUAL_INFEASIBLE,
 * SDP_MAX_ITER) or a negative error; `out` may be NULL. */
int sdp_solve(sdp_ctx* ctx, sdp_info* out);

/* Copy the last iterate out: X (n*n, the x iterate), y (m, equality
 * multipliers y_e), S (n*n, the dual slack -Y).  Any pointer may be NULL.
 * to_device != 0: the pointers are device memory. */
int sdp_get_solution(sdp_ctx* ctx, double* X, double* y, double* S, int to_device);

/* Copy the normalised infeasibility certificate of the last solve:
 * PRIMAL_INFEASIBLE -> cert_y (m) = y-bar_e and cert_M (n*n) = Y-bar;
 * DUAL_INFEASIBLE   -> cert_y zeroed and cert_M = x-bar.
 * Errors: SDP_E_STATE when the last solve found no certificate. */
int sdp_get_certificate(sdp_ctx* ctx, double* cert_y, double* cert_M, int to_device);

/* Standalone projection Pi_{S+}(W) (Eq. 2) by LOBPCG (Algorithm 3) from the
 * warm-start block V_warm (n x *m_inout, column-major, updated in place
 * with the final Ritz vectors; its buffer must hold n*mcap doubles).
 * `out` receives the n*n projection.  tol is the absolute residual-norm
 * tolerance per Ritz pair; tol <= 0 selects 0.5e-6*||W||_F/sqrt(2*m).
 * The mode (positive or negative eigenpairs) is chosen by the count rule
 * of Section 5 from the width of the warm-start block.  The context's
 * precision setting selects the product arithmetic.
 * Pointers are host memory unless on_device != 0.  The context needs no
 * sdp_setup.  Errors: SDP_E_INVALID, SDP_E_NUMERICAL, SDP_E_NOMEM. */
int sdp_project_psd(sdp_ctx* ctx, int n, const double* W, double* out, double* V_warm, int* m_inout,
                    int mcap, double tol, int on_device, sdp_proj_info* info);

/* The LOBPCG block product (Algorithm 3: A X, A R): out = W B for a
 * symmetric n x n W and an n x k block B, all column-major device arrays,
 * in the context's precision: SDP_PREC_FP64 on the CUDA cores, otherwise
 * split-BF16 x3 on the tcgen05 tensor cores with FP32 accumulation.
 * resplit_w = 0 reuses the bf16 split of the W passed last time (same n),
 * so repeated products with one W convert it once.  k <= ceil(n/3) + 2b.
 * Errors: SDP_E_INVALID, SDP_E_NOMEM, SDP_E_CUDA. */
int sdp_block_product(sdp_ctx* ctx, int n, const double* W, const double* B, int k, double* out, int resplit_w);

/* C = alpha op(A) op(B) + beta C for FP64 column-major device arrays of the
 * current device (op(X) = X, or X^T when trans_x != 0; op(A) is M x K,
 * op(B) K x N), computed on the tcgen05 tensor cores to FP64 accuracy by
 * the split-product scheme the mixed-precision Rayleigh-Ritz step uses for
 * its Grams, H = L^{-1} M L^{-T}, Ritz coefficients and block update
 * (Algorithm 2 inside Algorithm 3): each row of op(A) and column of op(B)
 * is scaled by a power of two and cut into six bf16 digit planes, the 21
 * leading digit products are accumulated exactly per 128-deep chunk, and
 * |C - op(A)op(B)| <= K 2^-44 max_k|A_mk| max_k|B_kn| elementwise (plus the
 * final rounding).  Inf/NaN inputs give NaN in the affected rows and
 * columns.  Runs on the context's stream and returns after it (the
 * context keeps a workspace, grown as needed; the context needs no
 * sdp_setup).  Errors: SDP_E_INVALID (sizes, leading dimensions),
 * SDP_E_NOMEM, SDP_E_CUDA, SDP_E_TIMEOUT (a bounded device wait gave up). */
int sdp_dense_product(sdp_ctx* ctx, int trans_a, int trans_b, int M, int N, int K, double alpha, const double* A,
                      int lda, const double* B, int ldb, double beta, double* C, int ldc);

/* Solve `count` set-up contexts together: every ADMM step of all of them is
 * issued as one batched launch sequence (one launch per kernel for the
 * whole group, each CTA finding its instance through a prefix map); the
 * LOBPCG loop is host-driven (its step count and subspace widths are read
 * back per step), so the sequence is not a CUDA graph.  All contexts
 * must share precision, rho, sigma, alpha, check_every and max_iter.
 * info (count entries) may be NULL.  Returns SDP_OK when every instance
 * finished (each info[k].status holds its own result). */
int sdp_batch_solve(int count, sdp_ctx* const* ctxs, sdp_info* info);

/* Continuous-batching server.  Requests are admitted while the resident
 * device state fits `hbm_budget_bytes` and at most `max_slots` are active;
 * every step advances all active requests by `iters_per_step` ADMM
 * iterations in one batched launch sequence; finished requests retire and
 * waiting ones are admitted between steps. */
int sdp_server_create(sdp_server** srv, const sdp_settings* settings, unsigned long long hbm_budget_bytes,
                      int max_slots, int iters_per_step, void* cuda_stream);
/* Queue a set-up context (ownership stays with the caller, who must keep
 * it alive until the ticket finishes). */
int sdp_server_submit(sdp_server* srv, sdp_ctx* ctx, unsigned long long* ticket);
/* Run one scheduling step: admit, advance, retire.  *n_active and
 * *n_queued (may be NULL) report the occupancy after the step. */
int sdp_server_step(sdp_server* srv, int* n_active, int* n_queued);
/* Status of a ticket: SDP_QUEUED, SDP_RUNNING or the final status; info
 * (may be NULL) is filled once the ticket is finished. */
int sdp_server_poll(sdp_server* srv, unsigned long long ticket, sdp_info* info);
void sdp_server_destroy(sdp_server* srv);

/* Device bytes a context of this size holds while resident (the server's
 * admission rule). */
unsigned long long sdp_footprint_bytes(int n, int m, long nnz, int precision);

/* Release every device buffer of the context. */
void sdp_destroy(sdp_ctx* ctx);

/* ---- projection of a small matrix without device allocation ------------
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory: code running while a CUDA stream is being
 * captured (cudaMalloc is not permitted there) and applications that pool
 * all device memory at start-up and forbid later allocation.
 *
 * out = Pi_{S+}(W) (Eq. 2) for a symmetric n x n W, both column-major
 * device arrays of the current device, computed by a one-CTA Jacobi
 * eigendecomposition on `cuda_stream` (NULL = legacy default stream).  The
 * call allocates nothing: its scratch (2 * n * n doubles) is a fixed
 * file-scope device array of 2 * SDP_NOALLOC_MAX_N^2 doubles (256 KiB)
 * that every GPU loading the library keeps until the process exits.
 *  - n > SDP_NOALLOC_MAX_N (or n < 1, NULL pointers): SDP_E_INVALID,
 *    nothing launched.
 *  - Every call looks up the current device's address of the scratch
 *    array (cudaGetSymbolAddress); the first call on a device may load the
 *    library's device code there, so make that first call before any
 *    stream capture begins.
 *  - Every call shares the one scratch array: calls that overlap on the
 *    GPU (different streams or host threads) race; serialise them.
 *  - W may equal out (in place): the kernel copies W into the scratch
 *    before it writes out.
 *  - Asynchronous: returns after the launch (SDP_OK, or SDP_E_CUDA when
 *    this call's launch failed; an error left pending by earlier work is
 *    neither reported nor cleared); synchronise the stream before reading
 *    `out`. */
#define SDP_NOALLOC_MAX_N 128
int sdp_project_psd_noalloc(int n, const double* W, double* out, void* cuda_stream);

/* Text of the last CUDA error seen by this thread (static storage). */
const char* sdp_last_error(void);

/* Limit, in seconds, of every bounded device wait of the library: the
 * tensor-core pipeline waits of the block product and the grid barriers of
 * the cooperative Rayleigh-Ritz and Jacobi kernels.  A wait that reaches it
 * gives up, the kernel skips the rest of its work after its own copies and
 * MMAs in flight have finished, and the call returns SDP_E_TIMEOUT with the
 * context still usable.  0 restores the default (2 s).  Process-wide; meant
 * for tests of the give-up path.  Errors: SDP_E_INVALID (negative or above
 * 60 s). */
int sdp_set_wait_limit(double seconds);

/* ---- instrumentation (no counterpart in the paper) ----------------------
 * Per kernel family: launches, device time between CUDA events recorded on
 * the launching stream around every launch of the family (only while
 * enabled), and the algorithmic flops / HBM bytes of those launches
 * (flops 2*n*n*k for an n x n by n x k product, bytes = operands read +
 * results written once).  Launch counts are kept always. */
typedef enum {
  SDP_PROF_PRODUCT = 0,  /* W times a block (LOBPCG A X, A R)          */
  SDP_PROF_GRAM = 1,     /* S^T S and S^T A S                         */
  SDP_PROF_RR = 2,       /* per-instance Rayleigh-Ritz (Chol, eig)    */
  SDP_PROF_UPDATE = 3,   /* new block S * Coef                        */
  SDP_PROF_RECON = 4,    /* Z = [W] + X Theta X^T, Y = rho (W - Z)    */
  SDP_PROF_RESID = 5,    /* residuals, compaction, random columns     */
  SDP_PROF_ADMM = 6,     /* linear step, relaxation                   */
  SDP_PROF_EXACT = 7,    /* full Jacobi eigendecomposition            */
  SDP_PROF_CHECK = 8,    /* termination / infeasibility reductions    */
  SDP_PROF_SPLIT = 9,    /* operand conversion for the tensor cores   */
  SDP_PROF_FAMILIES = 10
} sdp_prof_family;

typedef struct {
  long long launches;
  double ms;       /* summed event time of the timed launches */
  long long timed; /* launches that were timed                */
  double flops;
  double bytes;
} sdp_prof_entry;

/* on != 0: time every launch with CUDA events from now on. */
void sdp_prof_enable(int on);
/* zero every counter */
void sdp_prof_reset(void);
/* synchronise the pending events and copy one family's counters */
int sdp_prof_get(int family, sdp_prof_entry* out);
/* the same counters per named kernel (or named launch group), in name
 * order: entry idx (0-based) with its name copied into name[name_cap];
 * SDP_E_INVALID past the last one */
int sdp_prof_named(int idx, char* name, int name_cap, sdp_prof_entry* out);

#ifdef __cplusplus
}
#endif
#endif /* SDPGPU_H */
