// jacobi_kernels.cu -- the exact projection branch (Section 5: full
// eigendecomposition when the rank is between the thresholds, and at the
// first ADMM iteration): parallel cyclic Jacobi on the n x n matrix, one
// round of n/2 disjoint rotations per launch pair (angles, then the
// two-sided update of every 2x2 block plus the eigenvector update), then
// an ascending sort of the eigenpairs.  Batched over instances.
#include "common.cuh"
#include "kernels.h"

namespace sdpg {

__device__ __forceinline__ void jac_pair(int r, int k, int np, int* a, int* b) {
  if (k == 0) {
    *a = 0;
    *b = 1 + (r % (np - 1));
  } else {
    *a = 1 + (r + k) % (np - 1);
    *b = 1 + (r - k + (np - 1)) % (np - 1);
  }
}

// ||A||_F^2 of a rows x cols matrix in a fixed summation order (one CTA):
// the Jacobi threshold derived from it must not depend on scheduling, so
// that an instance gets bit-identical rotations alone and in a batch.
__device__ double cta_fro2_det(const double* A, int ld, int rows, int cols) {
  __shared__ double sh[1024];
  double part = 0.0;
  const long tot = (long)rows * cols;
  for (long t = threadIdx.x; t < tot; t += blockDim.x) {
    double a = A[idx2((int)(t % rows), (int)(t / rows), ld)];
    part += a * a;
  }
  sh[threadIdx.x] = part;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// ||W||_F^2 of each listed instance into ctl->jac_off (deterministic)
__global__ void k_fro2_det(Inst* insts, const int* list) {
  const Inst& I = insts[list[blockIdx.x]];
  double v = cta_fro2_det(I.W, I.ld, I.n, I.n);
  if (threadIdx.x == 0) I.ctl->jac_off = v;
}

__global__ void k_fro2_mat(const double* A, int ld, int rows, int cols, double* dst) {
  double v = cta_fro2_det(A, ld, rows, cols);
  if (threadIdx.x == 0) *dst = v;
}

// ||W||_F^2 into ctl->jac_off (to_w = 0) or ctl->wfro2 (to_w = 1)
__global__ void k_fro2(Inst* insts, WorkMap wm, int to_w) {
  __shared__ double sh[32];
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const size_t total = (size_t)I.ld * I.n;
  double part = 0.0;
  for (size_t q = (size_t)local * blockDim.x * 4 + threadIdx.x; q < total && q < (size_t)(local + 1) * blockDim.x * 4;
       q += blockDim.x) {
    if ((int)(q % I.ld) >= I.n) continue;
    double w = I.W[q];
    part += w * w;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    atomicAdd(to_w ? &I.ctl->wfro2 : &I.ctl->jac_off, s);
  }
}

// E = (negate ? -W : W), EV = I
__global__ void k_jac_init(Inst* insts, WorkMap wm, int negate) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const size_t total = (size_t)I.ld * I.n;
  for (size_t q = (size_t)local * blockDim.x * 4 + threadIdx.x; q < total && q < (size_t)(local + 1) * blockDim.x * 4;
       q += blockDim.x) {
    int i = (int)(q % I.ld), j = (int)(q / I.ld);
    if (i >= I.n) continue;
    I.E[q] = negate ? -I.W[q] : I.W[q];
    I.EV[q] = (i == j) ? 1.0 : 0.0;
  }
}

// rotation angles of round `round` (symmetric Schur 2x2, Golub & Van Loan 8.5.2)
__global__ void k_jac_angles(Inst* insts, WorkMap wm, int round) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const int n = I.n, np = n + (n & 1), P2 = np / 2;
  if (round >= np - 1) return;
  const int k = local * blockDim.x + threadIdx.x;
  if (k >= P2) return;
  int a, b;
  jac_pair(round, k, np, &a, &b);
  double c = 1.0, s = 0.0;
  if (a < n && b < n) {
    double thr = kJacobiAbs64 * sqrt(I.ctl->jac_off) / (double)n;
    double hab = I.E[idx2(a, b, I.ld)];
    double haa = I.E[idx2(a, a, I.ld)], hbb = I.E[idx2(b, b, I.ld)];
    if (jacobi_rotates(hab, haa, hbb, kJacobiRel64, thr)) {
      double tau = (hbb - haa) / (2.0 * hab);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      s = t * c;
      atomicAdd(&I.ctl->jac_rot, 1);
    }
  }
  I.erot[2 * k] = c;
  I.erot[2 * k + 1] = s;
}

// two-sided update of all 2x2 blocks of E and column rotations of EV
__global__ void k_jac_apply(Inst* insts, WorkMap wm, int round) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const int n = I.n, np = n + (n & 1), P2 = np / 2, ld = I.ld;
  if (round >= np - 1) return;
  const long e = (long)local * blockDim.x + threadIdx.x;
  const long nblk = (long)P2 * P2;
  if (e < nblk) {
    int ki = (int)(e % P2), kj = (int)(e / P2);
    int ai, bi, aj, bj;
    jac_pair(round, ki, np, &ai, &bi);
    jac_pair(round, kj, np, &aj, &bj);
    double ci = I.erot[2 * ki], si = I.erot[2 * ki + 1], cj = I.erot[2 * kj], sj = I.erot[2 * kj + 1];
    if (si == 0.0 && sj == 0.0) return;
    bool vai = ai < n, vbi = bi < n, vaj = aj < n, vbj = bj < n;
    double haa = (vai && vaj) ? I.E[idx2(ai, aj, ld)] : 0.0;
    double hab = (vai && vbj) ? I.E[idx2(ai, bj, ld)] : 0.0;
    double hba = (vbi && vaj) ? I.E[idx2(bi, aj, ld)] : 0.0;
    double hbb = (vbi && vbj) ? I.E[idx2(bi, bj, ld)] : 0.0;
    double taa = cj * haa - sj * hab, tab = sj * haa + cj * hab;
    double tba = cj * hba - sj * hbb, tbb = sj * hba + cj * hbb;
    double naa = ci * taa - si * tba, nba = si * taa + ci * tba;
    double nab = ci * tab - si * tbb, nbb = si * tab + ci * tbb;
    if (ki == kj && si != 0.0) { nab = 0.0; nba = 0.0; }
    if (vai && vaj) I.E[idx2(ai, aj, ld)] = naa;
    if (vai && vbj) I.E[idx2(ai, bj, ld)] = nab;
    if (vbi && vaj) I.E[idx2(bi, aj, ld)] = nba;
    if (vbi && vbj) I.E[idx2(bi, bj, ld)] = nbb;
  } else {
    long f = e - nblk;
    if (f >= (long)n * P2) return;
    int row = (int)(f % n), k = (int)(f / n);
    double c = I.erot[2 * k], s = I.erot[2 * k + 1];
    if (s == 0.0) return;
    int a, b;
    jac_pair(round, k, np, &a, &b);
    if (a >= n || b >= n) return;
    double ua = I.EV[idx2(row, a, ld)], ub = I.EV[idx2(row, b, ld)];
    I.EV[idx2(row, a, ld)] = c * ua - s * ub;
    I.EV[idx2(row, b, ld)] = s * ua + c * ub;
  }
}

// eigenvalues (diag of E) in ascending order: elam[0..n) sorted, elam[n..2n)
// their negatives, eord the permutation; counts of positive/negative ones
// in ctl->npos / ctl->npos_rr (negative count).
__global__ void k_jac_sort(Inst* insts, const int* list) {
  const Inst& I = insts[list[blockIdx.x]];
  const int n = I.n, ld = I.ld;
  __shared__ int np, nn;
  if (threadIdx.x == 0) { np = 0; nn = 0; }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double li = I.E[idx2(i, i, ld)];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = I.E[idx2(j, j, ld)];
      rank += rank_before((double)lj, j, (double)li, i);
    }
    I.eord[rank] = i;
    if (li > 0.0) atomicAdd(&np, 1);
    else if (li < 0.0) atomicAdd(&nn, 1);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double l = I.E[idx2(I.eord[r], I.eord[r], ld)];
    I.elam[r] = l;
    I.elam[n + r] = -l;
  }
  if (threadIdx.x == 0) {
    I.ctl->npos = np;
    I.ctl->npos_rr = nn;
  }
}

// E[:, r] = EV[:, eord[r]] (sorted eigenvectors)
__global__ void k_jac_gather(Inst* insts, WorkMap wm) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const int r = local;
  if (r >= I.n) return;
  const double* src = I.EV + (size_t)I.eord[r] * I.ld;
  double* dst = I.E + (size_t)r * I.ld;
  for (int i = threadIdx.x; i < I.n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace sdpg

namespace sdpg {
// Seed the LOBPCG block from the sorted eigenvectors in E: ctl->mode is
// the next mode and ctl->m the block width.  POS: the m largest
// eigenvectors of W in ascending order; NEG: the m largest of -W.
__global__ void k_seed_block(Inst* insts, WorkMap wm) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const Ctl* c = I.ctl;
  const int j = local, m = c->m, n = I.n;
  if (j >= m || c->mode == MODE_EXACT) return;
  int src = (c->mode == MODE_POS) ? (n - m + j) : (m - 1 - j);
  const double* s = I.E + (size_t)src * I.ld;
  double* d = I.S[I.par] + (size_t)j * I.ld;
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__global__ void k_copy_cols(const double* src, int lds, double* dst, int ldd, int rows, int cols, double scale) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * cols) return;
  int i = (int)(t % rows), j = (int)(t / rows);
  dst[(size_t)i + (size_t)j * ldd] = scale * src[(size_t)i + (size_t)j * lds];
}
}  // namespace sdpg
