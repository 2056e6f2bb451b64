// rr_blocked.cu -- blocked pieces of the wide Rayleigh-Ritz step (Algorithm
// 2 inside Algorithm 3) whose O(p^3) work runs as FP64-accurate tensor-core
// products (oz_gemm.cu), driven from the host:
//
//  * Cholesky factorisation and inverse of a Gram matrix, G = L L^T, in
//    diagonal blocks of kBlk columns: the kBlk x kBlk diagonal block is
//    factored and inverted by one CTA in shared memory (k_potrf_inv_block,
//    FP64), the panel below it (L21 = G21 L11^{-T}) and the trailing update
//    (G22 -= L21 L21^T) are products, and L^{-1} is assembled block row by
//    block row, L^{-1}[i, :i] = -L_ii^{-1} (L[i, :i] L^{-1}[:i, :i]);
//  * the back-transform of the tridiagonal eigenvectors, Y = Q Z with
//    Q = P_0 P_1 ... P_{p-3} the Householder reflectors of the reduction,
//    with kBlk reflectors at a time in compact WY form I - V T V^T
//    (k_wy_vmat writes V, k_wy_tmat the triangular T from V^T V and the
//    tau of the reflectors), applied as Y -= V (T (V^T Y)).
#include "kernels.h"
#include "gridbar.cuh"

namespace sdpg {

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA: the bb x bb diagonal block of G at (j0, j0) (bb <= kBlk): its
// Cholesky factor L11 (lower, written back into G with zeros above) and
// L11^{-1} (written into Linv's diagonal block).  A pivot d <= piv_min (the
// Schur complement's diagonal before the square root) records the 1-based
// column in bar->fail; the block is then left as it is.  The inverse is
// formed by forward substitution, one column per warp (lanes split each dot
// product), into the upper triangle of the shared block (transposed).
// Dynamic shared memory: potrf_block_smem(BLK) bytes.
template <int BLK>
__global__ void __launch_bounds__(1024) k_potrf_inv_block(double* G, int ldg, double* Linv, int ldl, int j0, int bb,
                                                          double piv_min, GridBar* bar) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double (*A)[BLK + 1] = (double (*)[BLK + 1])smraw;
  __shared__ double xd[BLK];
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (*(volatile int*)&bar->fail || *(volatile int*)&bar->err) return;
  for (int t = tid; t < bb * bb; t += nt) {
    const int i = t % bb, j = t / bb;
    A[i][j] = i >= j ? G[(size_t)(j0 + i) + (size_t)(j0 + j) * ldg] : 0.0;
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  // right-looking Cholesky of the block
  // (the pivot's square root and reciprocal by one thread: an SM issues only
  // about two FP64 operations per clock, so redundant FP64 work is costly)
  __shared__ double s_inv;
  for (int j = 0; j < bb; ++j) {
    const double d = A[j][j];
    if (!(d > piv_min)) {
      if (tid == 0) fail = j0 + j + 1;
      break;  // uniform: every thread read the same pivot
    }
    __syncthreads();
    if (tid == 0) {
      const double sq = sqrt(d);
      A[j][j] = sq;
      s_inv = 1.0 / sq;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int r = j + 1 + tid; r < bb; r += nt) A[r][j] *= inv;
    __syncthreads();
    for (int c = j + 1 + wid; c < bb; c += nw) {
      const double lc = A[c][j];
      for (int r = c + lane; r < bb; r += 32) A[r][c] -= A[r][j] * lc;
    }
    __syncthreads();
  }
  __syncthreads();
  if (fail) {
    if (tid == 0) atomicCAS(&bar->fail, 0, fail);
    return;
  }
  for (int t = tid; t < bb * bb; t += nt) {
    const int i = t % bb, j = t / bb;
    G[(size_t)(j0 + i) + (size_t)(j0 + j) * ldg] = i >= j ? A[i][j] : 0.0;
  }
  for (int j = tid; j < bb; j += nt) xd[j] = 1.0 / A[j][j];
  __syncthreads();
  // X = L^{-1}: column j solves L x = e_j by forward substitution in axpy
  // form, one column per warp: once x_k is known, the rows below take
  // -L_ik x_k (lane-parallel FMAs, no reductions -- an FP64 warp instruction
  // costs the SM's FP64 pipe tens of cycles).  X[i][j] is kept at A[j][i].
  for (int j = wid; j < bb; j += nw) {
    double acc[BLK / 32];  // running sums of the rows this lane owns: rows i = lane + 32 q
#pragma unroll
    for (int q = 0; q < BLK / 32; ++q) acc[q] = 0.0;
    for (int k = j; k < bb; ++k) {
      // x_k = (delta_jk - sum_{j <= l < k} L_kl x_l) / L_kk, held by the lane owning row k
      double xk = 0.0;
      double ak = 0.0;
#pragma unroll
      for (int q = 0; q < BLK / 32; ++q)  // register select, no local-memory indexing
        if (q == (k >> 5)) ak = acc[q];
      if (lane == (k & 31)) xk = ((k == j ? 1.0 : 0.0) - ak) * xd[k];
      xk = __shfl_sync(0xffffffffu, xk, k & 31);
      if (lane == 0) A[j][k] = xk;  // diagonal entry too (overwritten with xd below)
#pragma unroll
      for (int q = 0; q < BLK / 32; ++q) {
        const int i = lane + 32 * q;
        if (i > k && i < bb) acc[q] += A[i][k] * xk;
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < bb * bb; t += nt) {
    const int i = t % bb, j = t / bb;
    Linv[(size_t)(j0 + i) + (size_t)(j0 + j) * ldl] = i > j ? A[j][i] : (i == j ? xd[i] : 0.0);
  }
}

template __global__ void k_potrf_inv_block<kPotrfBlk>(double*, int, double*, int, int, int, double, GridBar*);

// V (p x nref, ld p): column k = the Householder vector of reflector k
// (zero above row k+1, one at row k+1, below it the vector stored in
// column k of the reduced matrix A, ld p), for k < nref
__global__ void k_wy_vmat(const double* A, int p, int nref, double* V) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p * nref) return;
  const int i = (int)(t % p), k = (int)(t / p);
  V[t] = i < k + 1 ? 0.0 : (i == k + 1 ? 1.0 : A[(size_t)k * p + i]);
}

// One CTA per block of kBlk reflectors [k0, k0 + bb): T (bb x bb, upper,
// ld kBlk) with P_k0 ... P_{k0+bb-1} = I - V T V^T, from Gv = V^T V of the
// block (bb x bb, ld kBlk, in place) and tau: T_ii = tau_i and
// T[0:i, i] = -tau_i T[0:i, 0:i] Gv[0:i, i].
// Dynamic shared memory: kBlkSmem bytes.
__global__ void __launch_bounds__(256) k_wy_tmat(double* Tall, const double* tau, int nref) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double (*Tm)[kBlk + 1] = (double (*)[kBlk + 1])smraw;
  __shared__ double z[kBlk];
  const int blk = blockIdx.x, k0 = blk * kBlk, bb = min(kBlk, nref - k0);
  const int tid = threadIdx.x, nt = blockDim.x;
  double* T = Tall + (size_t)blk * kBlk * kBlk;
  if (bb <= 0) return;
  for (int t = tid; t < kBlk * kBlk; t += nt) Tm[t % kBlk][t / kBlk] = 0.0;
  __syncthreads();
  for (int i = 0; i < bb; ++i) {
    const double ti = tau[k0 + i];
    for (int r = tid; r < i; r += nt) z[r] = T[r + (size_t)i * kBlk];  // Gv[r, i]
    __syncthreads();
    for (int r = tid; r < i; r += nt) {
      double acc = 0.0;
      for (int c = r; c < i; ++c) acc += Tm[r][c] * z[c];
      Tm[r][i] = -ti * acc;
    }
    if (tid == 0) Tm[i][i] = ti;
    __syncthreads();
  }
  for (int t = tid; t < kBlk * kBlk; t += nt) {
    const int r = t % kBlk, c = t / kBlk;
    T[t] = (r < bb && c < bb) ? Tm[r][c] : 0.0;
  }
}

}  // namespace sdpg
