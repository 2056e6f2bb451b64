// common.cuh -- device data structures shared by the sdpgpu kernels.
//
// One SDP instance (min <C,X> s.t. A(X) = b, X psd) owns a set of device
// buffers described by `Inst`; its LOBPCG/ADMM control state lives in `Ctl`.
// Kernels are batched over a group of instances: a launch covers the work
// units of every instance, found through a per-launch prefix array
// (`WorkMap`), so a single solve, a batch and the server run the same code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sdpg {

enum { MODE_POS = 0, MODE_NEG = 1, MODE_EXACT = 2 };

// Jacobi rotation rule: rotate the pair (a, b) only while
//   |h_ab| > max(rel * sqrt(|h_aa h_bb|), abs_thr),  abs_thr = eps ||H||_F / n
// with rel = 0: the off-diagonal Frobenius norm left is below eps ||H||_F.
// A relative rule (rel > 0) leaves eigenvectors inside clusters of close
// Ritz values too inaccurate for the per-pair residual test of LOBPCG, so
// it is not used.  A sweep without rotations ends the iteration.
constexpr double kJacobiRel64 = 0.0, kJacobiAbs64 = 4e-16;
constexpr double kJacobiRel32 = 0.0, kJacobiAbs32 = 4e-7;
__device__ __forceinline__ bool jacobi_rotates(double hab, double haa, double hbb, double rel, double abs_thr) {
  double t = rel * sqrt(fabs(haa * hbb));
  return fabs(hab) > (t > abs_thr ? t : abs_thr);
}

// Strict total order for the rank sort of Ritz values / eigenvalues: NaN
// sorts below every number (it is never among the selected top values) and
// ties break by index, so the ranks of p values always form a permutation of
// 0..p-1 and every slot of the order array is written exactly once.
__device__ __forceinline__ bool rank_before(double lj, int j, double li, int i) {
  const bool nj = lj != lj, ni = li != li;
  if (nj != ni) return nj;
  if (!nj && lj != li) return lj < li;
  return j < i;
}

// Per-instance control block (device memory, read back by the host).
// Bounded device waits give up after this much elapsed time (globaltimer
// nanoseconds) unless a shorter limit is set for a test of the expiry path.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// Clean-up waits after a give-up (outstanding copies and MMAs must finish
// before a CTA releases its shared and tensor memory) use this limit.
constexpr unsigned long long kDrainLimitNs = 4000000000ull;
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Ctl {
  int mode;      // projection mode of the current ADMM iteration
  int m;         // LOBPCG block width
  int mP;        // columns of Delta X in the trial subspace
  int nfresh;    // trailing random columns of the block (not Ritz vectors yet)
  int active;    // 1 while LOBPCG iterates on this instance
  int p;         // trial-subspace width of the pending Rayleigh-Ritz step
  int keep;      // Ritz pairs the pending Rayleigh-Ritz step keeps
  int npos;      // positive Ritz values in the block
  int npos_rr;   // positive Ritz values of the last Rayleigh-Ritz step
  int rr_fail;   // Cholesky-QR breakdown in the last Rayleigh-Ritz step
  int jac_rot;   // rotations in the last Jacobi sweep (exact branch)
  int chol_fail; // cone test (Cholesky) result: 0 positive definite
  int sweeps;
  int snap;      // 1: keep x, Y, y_e of this iteration (termination check follows)
  int ma;        // residual columns still active (not yet within tol)
  int mPa;       // Delta X columns of active Ritz pairs
  int soft_lock; // 1: pairs within tol leave R and Delta X of the next step
  int spare_;
  double tol;    // LOBPCG residual tolerance
  double res_max;  // largest Ritz residual norm of the block
  double res_pos2; // sum of squared residual norms of the positive pairs
  double jac_off;  // off-diagonal norm^2 (exact branch)
  double wfro2;    // ||W||_F^2 of the matrix being projected (mixed precision)
  double thmin;    // smallest |Ritz value| of the block (mixed precision)
};

// Per-instance reduction results of the termination check (Section 5).
struct Check {
  double rp_dense;   // max |x - Z|
  double rp_cons;    // max |A(x) - b|
  double rd_dense;   // max |C + Y| over positions outside the sparsity of A
  double rd_sparse;  // max |C + Y + A^T y| over positions of A
  double nx, nz, nC, nY;  // inf-norms for the relative tolerances
  double obj;        // <C, x>
  double ndy_e;      // max |y - yprev|
  double ndY;        // max |Y - Yprev|
  double at_dense;   // max |dY| outside the sparsity of A
  double at_sparse;  // max |dY + A^T dy| on the sparsity of A
  double bdy;        // b^T dy
  double ndx;        // max |x - xprev|
  double adx;        // max |A(dx)|
  double cdx;        // <C, dx>
  double nAx;        // max |A(x)|
  double nATy;       // max |A^T y + Y| (dual scale)
};

struct Inst {
  int n, ld;          // size and leading dimension of every n x n array
  int mc;             // number of equality constraints
  int nent;           // distinct sparse positions (i <= j) touched by A
  int mcap, bexp;     // LOBPCG block capacity and expansion width
  int pcap;           // trial-subspace capacity (3*mcap)
  int nF;             // Schur block of K (dense)
  double rho, sigma, alpha;
  // dense state, ld x n, FP64
  double *C, *x, *Z, *Y, *W, *xprev, *Yprev;
  // constraint vectors (mc)
  double *b, *ye, *ze, *yeprev, *u, *v, *tv;
  // sparse structure: entry -> (constraints, values); constraint -> (entries, weights)
  int *ent_i, *ent_j, *ent_ptr, *ent_con;
  double *ent_val, *ent_r, *ent_corr;
  int *con_ptr, *con_ent;
  double* con_w;
  uint32_t* smask;    // bit (i + j*ld) set when (i,j) is a sparse position
  // K = s I + rho A A^T eliminated by blocks: D diagonal, F dense Schur
  double* kdiag;      // mc
  int *isD, *fpos, *Flist;
  int *k_ptr, *k_col;  // off-diagonal K entries (CSR)
  double* k_val;
  double* Lf;         // nF x nF lower Cholesky factor of the Schur complement
  // LOBPCG workspace (FP64 storage; the compute precision is a launch choice)
  double *S[2], *AS[2]; // ld x pcap: [X | R | dX] and [AX | AR | AdX]
  int par;              // which of S/AS holds the current block
  double *G, *M, *Linv, *H, *U;  // pcap x pcap
  double *Coef;         // pcap x mcap
  double *theta;        // mcap (Ritz values of the block, ascending)
  double *resn;         // pcap (residual norms / column norms)
  int *slot;            // mcap: compacted position of each active column (-1: locked)
  double *gpart;        // Gram split-K partials
  // exact branch (full Jacobi)
  double *E, *EV, *elam, *erot;  // E, EV ld x n; elam n; erot 2*n (c,s per pair)
  int* eord;            // n (ascending order)
  // mixed precision operands (bf16 hi/lo of W and of the multiplied block)
  void *Whi, *Wlo, *Bhi, *Blo;
  float* Wf;            // FP32 copy of W (mixed mode reconstruction operand)
  float* tcpart;        // split-K partials of the tensor-core product (8 x ld x mcap)
  Ctl* ctl;
  Check* chk;
  double* chk_part;     // per-CTA partials of the check
  int prec;             // sdp_precision
  int piv_loose;        // 1: Cholesky-QR pivots below 1e-6 count as breakdown (the trial subspace's
                        // products, hence S^T A S, carry split-BF16 or FP32 errors), else 1e-12
};

// State of a grid-wide barrier and of the cooperative kernels using it.
struct GridBar {
  unsigned count, gen;
  unsigned top;        // groups arrived (two-level barrier)
  unsigned grp[64];    // CTAs arrived per group of 16
  int err;     // a barrier wait gave up (bounded wait)
  int fail;    // Cholesky breakdown column (1-based), 0 if none
  int sweeps;  // Jacobi sweeps done
  int pad;
  unsigned long long limit_ns;  // wait limit of gbar (0: kWaitLimitNs)
  double fro2; // ||H||_F^2
  int rot[64]; // rotations per sweep
};

// Prefix map from a flat block index to (instance, local unit).
struct WorkMap {
  const int* prefix;  // count+1 entries, prefix[0] = 0
  int count;
};

__device__ __forceinline__ int find_inst(const WorkMap& w, int blk, int* local) {
  int lo = 0, hi = w.count;  // prefix[lo] <= blk < prefix[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (w.prefix[mid] <= blk) lo = mid;
    else hi = mid;
  }
  *local = blk - w.prefix[lo];
  return lo;
}

__device__ __forceinline__ size_t idx2(int i, int j, int ld) { return (size_t)i + (size_t)j * (size_t)ld; }

// High 32 bits of a 32 x 32-bit product (the hardware instruction on the
// device; host builds are for the CPU tests of the device helpers).
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Philox4x32-10 (Salmon et al., SC'11): the counter-based generator of the
// random expansion columns.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = mulhi32(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    uint32_t hi1 = mulhi32(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// Standard normal deviate for (row, col) of random draw `draw` of stream
// `stream`: two 53-bit uniforms from one Philox block, Box-Muller.
__device__ __forceinline__ double philox_normal(unsigned long long seed, uint32_t stream, uint32_t draw,
                                                uint32_t row, uint32_t col) {
  uint32_t c[4] = {row, col, draw, stream};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  unsigned long long a = ((((unsigned long long)c[0]) << 32) | c[1]) >> 11;
  unsigned long long b = ((((unsigned long long)c[2]) << 32) | c[3]) >> 11;
  double u1 = ((double)a + 1.0) * (1.0 / 9007199254740992.0);
  double u2 = (double)b * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // IEEE-754 ordering of non-negative doubles equals that of their bit patterns
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace sdpg
