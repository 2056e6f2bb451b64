// rr_large.cu -- Rayleigh-Ritz (Algorithm 2) for wide trial subspaces,
// spread over every SM: cooperative kernels with a grid barrier for the
// Cholesky factorisation G = L L^T and the triangular inverse L^{-1}
// (Cholesky QR, Section 4), and for the symmetric eigendecomposition by
// parallel cyclic Jacobi (also the exact projection of Section 1 / Eq. 2).
// H = L^{-1} M L^{-T} and Coef = L^{-T} U are batched GEMM launches.
//
// Grid barrier: generation counter; every wait is bounded (about a
// second); on expiry the kernel records SDP_E_TIMEOUT-style status in
// GridBar::err and returns.  Launched with cudaLaunchCooperativeKernel,
// so all CTAs are co-resident and the bound is never reached in normal
// operation.
#include "common.cuh"
#include "kernels.h"
#include "gridbar.cuh"

namespace sdpg {


// ---------------------------------------------------------------------------
// Blocked Cholesky (32-column panels) and triangular inverse, in place on
// G (lower triangle receives L), Linv = L^{-1}.  A pivot below piv_min
// (Gram of unit-norm columns) reports breakdown in b->fail (1-based col).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_inv_coop(double* G, double* Linv, int p, double piv_min, GridBar* b) {
  __shared__ T Lkk[32][33];
  __shared__ int fail;
  const int nb = (p + 31) / 32;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int kb = 0; kb < nb; ++kb) {
    const int c0 = kb * 32, w = min(32, p - c0);
    // diagonal block factored redundantly by every CTA (tiny)
    for (int t = tid; t < 32 * 32; t += nthr) {
      int i = t % 32, j = t / 32;
      Lkk[i][j] = (i < w && j < w) ? (T)G[idx2(c0 + i, c0 + j, p)] : (T)0;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    if (tid < 32) {  // one warp: right-looking Cholesky of the w x w block
      for (int j = 0; j < w; ++j) {
        T d = __shfl_sync(0xffffffffu, Lkk[j][j], 0);
        if (tid == 0) {
          if (!(d > (T)piv_min)) fail = c0 + j + 1;
          Lkk[j][j] = sqrt(d > (T)0 ? d : (T)1);
        }
        __syncwarp();
        T ljj = Lkk[j][j];
        if (tid > j && tid < w) Lkk[tid][j] /= ljj;
        __syncwarp();
        for (int k = j + 1; k < w; ++k)
          if (tid >= k && tid < w) Lkk[tid][k] -= Lkk[tid][j] * Lkk[k][j];
        __syncwarp();
      }
    }
    __syncthreads();
    if (fail) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(&b->fail, 0, fail);
      return;  // every CTA sees the same block and returns here
    }
    // panel: rows below, L_ik = A_ik L_kk^{-T}
    for (int i = c0 + w + blockIdx.x * nthr + tid; i < p; i += gridDim.x * nthr) {
      T l[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= w) break;
        T acc = (T)G[idx2(i, c0 + j, p)];
        for (int t = 0; t < j; ++t) acc -= l[t] * Lkk[j][t];
        l[j] = acc / Lkk[j][j];
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= w) break;
        G[idx2(i, c0 + j, p)] = (double)l[j];
      }
    }
    if (!gbar(b)) return;
    // every CTA is past its read of the diagonal block: store L_kk
    if (blockIdx.x == 0)
      for (int t = tid; t < w * w; t += nthr) {
        int i = t % w, j = t / w;
        G[idx2(c0 + i, c0 + j, p)] = i >= j ? (double)Lkk[i][j] : 0.0;
      }
    // trailing update of the lower triangle
    const int r0 = c0 + w, tw = p - r0;
    const long tot = (long)tw * tw;
    for (long e = (long)blockIdx.x * nthr + tid; e < tot; e += (long)gridDim.x * nthr) {
      int i = r0 + (int)(e % tw), j = r0 + (int)(e / tw);
      if (i < j) continue;
      T acc = 0;
      for (int t = 0; t < w; ++t) acc += (T)G[idx2(i, c0 + t, p)] * (T)G[idx2(j, c0 + t, p)];
      G[idx2(i, j, p)] = (double)((T)G[idx2(i, j, p)] - acc);
    }
    if (!gbar(b)) return;
  }
  // Linv = L^{-1}: block rows in order; block row k of column c needs block
  // rows < k of the same column.
  for (int kb = 0; kb < nb; ++kb) {
    const int c0 = kb * 32, w = min(32, p - c0);
    for (int t = tid; t < 32 * 32; t += nthr) {
      int i = t % 32, j = t / 32;
      Lkk[i][j] = (i < w && j < w) ? (T)G[idx2(c0 + i, c0 + j, p)] : (T)0;
    }
    __syncthreads();
    // each warp handles one column c at a time; lane r = row c0 + r
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    for (int c = blockIdx.x * nw + warp; c < p; c += gridDim.x * nw) {
      T rhs = 0;
      if (lane < w) {
        int row = c0 + lane;
        rhs = (row == c) ? (T)1 : (T)0;
        if (c < c0)
          for (int q = c; q < c0; ++q) rhs -= (T)G[idx2(row, q, p)] * (T)Linv[idx2(q, c, p)];
      }
      // forward substitution with Lkk across the warp
      T x = 0;
      for (int j = 0; j < w; ++j) {
        T s = (lane == j) ? rhs : (T)0;
        // x_j = (rhs_j - sum_{t<j} Lkk[j][t] x_t) / Lkk[j][j]
        T contrib = (lane < j) ? Lkk[j][lane] * x : (T)0;
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
        contrib = __shfl_sync(0xffffffffu, contrib, 0);
        T rj = __shfl_sync(0xffffffffu, rhs, j);
        T xj = (rj - contrib) / Lkk[j][j];
        if (lane == j) x = xj;
        (void)s;
      }
      if (lane < w) Linv[idx2(c0 + lane, c, p)] = (c <= c0 + lane) ? (double)x : 0.0;
    }
    if (!gbar(b)) return;
  }
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi (round-robin ordering) across the grid, with H
// double-buffered (H -> H2 -> H ...) so that each round reads only
// pre-round values and needs a single grid barrier.  U accumulates the
// rotations (set to I here).  The result ends in H (copied back if the
// last round wrote H2).  b->rot[s] counts rotations of sweep s (zeroed by
// the host); *fro2 = ||H||_F^2 computed beforehand in a fixed order; the
// rotation rule is jacobi_rotates(rel, abs_eps * ||H||_F / p).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void jac_angle(const double* H, int ldh, int a, int bb, int p, double thr, double rel, T* c,
                                          T* s) {
  *c = (T)1;
  *s = (T)0;
  if (a >= p || bb >= p) return;
  T hab = (T)H[idx2(a, bb, ldh)];
  T haa = (T)H[idx2(a, a, ldh)], hbb = (T)H[idx2(bb, bb, ldh)];
  if (!jacobi_rotates((double)hab, (double)haa, (double)hbb, rel, thr)) return;
  T tau = (hbb - haa) / ((T)2 * hab);
  T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
  *c = (T)1 / sqrt((T)1 + t * t);
  *s = t * *c;
}

__device__ __forceinline__ void rr_pair2(int r, int k, int np, int* a, int* b) {
  if (k == 0) {
    *a = 0;
    *b = 1 + (r % (np - 1));
  } else {
    *a = 1 + (r + k) % (np - 1);
    *b = 1 + (r - k + (np - 1)) % (np - 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_jacobi_coop(double* H, double* H2, int ldh, double* U, int ldu, int p,
                                                     double rel, double abs_eps, int max_sweeps, const double* fro2,
                                                     GridBar* b) {
  // per round: every CTA computes the round's P2 rotations into shared
  // memory, then updates the 2x2 blocks of its own block-columns kj (all
  // block-rows ki) and the matching columns of U.
  extern __shared__ __align__(16) unsigned char jsm[];
  const int np = p + (p & 1), P2 = np / 2;
  T* cc = (T*)jsm;
  T* ss = cc + P2;
  int* pa = (int*)(ss + P2);
  int* pb = pa + P2;
  __shared__ int nrot;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long gthreads = (long)gridDim.x * nt, gt = (long)blockIdx.x * nt + tid;
  if (*(volatile int*)&b->fail || *(volatile int*)&b->err) return;
  for (long t = gt; t < (long)p * p; t += gthreads) {
    int i = (int)(t % p), j = (int)(t / p);
    U[idx2(i, j, ldu)] = (i == j) ? 1.0 : 0.0;
  }
  if (!gbar(b)) return;
  const double thr = abs_eps * sqrt(*fro2) / (double)(p > 0 ? p : 1);
  double* src = H;
  double* dst = H2;
  if (blockIdx.x == 0 && tid == 0) b->sweeps = 0;
  if (p >= 2) {
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      for (int r = 0; r < np - 1; ++r) {
        if (tid == 0) nrot = 0;
        __syncthreads();
        for (int k = tid; k < P2; k += nt) {
          int a, bb;
          rr_pair2(r, k, np, &a, &bb);
          T c, s;
          jac_angle<T>(src, ldh, a, bb, p, thr, rel, &c, &s);
          cc[k] = c;
          ss[k] = s;
          pa[k] = a;
          pb[k] = bb;
          if (s != (T)0) atomicAdd(&nrot, 1);
        }
        __syncthreads();
        if (blockIdx.x == 0 && tid == 0 && nrot) atomicAdd(&b->rot[sweep], nrot);
        for (int kj = blockIdx.x; kj < P2; kj += gridDim.x) {
          const int aj = pa[kj], bj = pb[kj];
          const T cj = cc[kj], sj = ss[kj];
          const bool vaj = aj < p, vbj = bj < p;
          for (int ki = tid; ki < P2; ki += nt) {
            const int ai = pa[ki], bi = pb[ki];
            const T ci = cc[ki], si = ss[ki];
            const bool vai = ai < p, vbi = bi < p;
            T haa = (vai && vaj) ? (T)src[idx2(ai, aj, ldh)] : (T)0;
            T hab = (vai && vbj) ? (T)src[idx2(ai, bj, ldh)] : (T)0;
            T hba = (vbi && vaj) ? (T)src[idx2(bi, aj, ldh)] : (T)0;
            T hbb = (vbi && vbj) ? (T)src[idx2(bi, bj, ldh)] : (T)0;
            T taa = cj * haa - sj * hab, tab = sj * haa + cj * hab;
            T tba = cj * hba - sj * hbb, tbb = sj * hba + cj * hbb;
            T naa = ci * taa - si * tba, nba = si * taa + ci * tba;
            T nab = ci * tab - si * tbb, nbb = si * tab + ci * tbb;
            if (ki == kj && si != (T)0) { nab = (T)0; nba = (T)0; }
            if (vai && vaj) dst[idx2(ai, aj, ldh)] = (double)naa;
            if (vai && vbj) dst[idx2(ai, bj, ldh)] = (double)nab;
            if (vbi && vaj) dst[idx2(bi, aj, ldh)] = (double)nba;
            if (vbi && vbj) dst[idx2(bi, bj, ldh)] = (double)nbb;
          }
          if (sj != (T)0 && vaj && vbj) {
            for (int row = tid; row < p; row += nt) {
              T ua = (T)U[idx2(row, aj, ldu)], ub = (T)U[idx2(row, bj, ldu)];
              U[idx2(row, aj, ldu)] = (double)(cj * ua - sj * ub);
              U[idx2(row, bj, ldu)] = (double)(sj * ua + cj * ub);
            }
          }
        }
        if (!gbar(b)) return;
        double* tmp = src;
        src = dst;
        dst = tmp;
      }
      if (blockIdx.x == 0 && tid == 0) b->sweeps = sweep + 1;
      if (*(volatile int*)&b->rot[sweep] == 0) break;
    }
  }
  if (src != H) {
    for (long t = gt; t < (long)p * p; t += gthreads) {
      int i = (int)(t % p), j = (int)(t / p);
      H[idx2(i, j, ldh)] = src[idx2(i, j, ldh)];
    }
  }
}

// Ascending order of the diagonal of H (rank sort), the top `keep` values,
// positive count; grid over i.
__global__ void k_diag_rank(const double* H, int ldh, int p, int* ord, int* fail) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  double li = H[idx2(i, i, ldh)];
  if (!isfinite(li)) atomicCAS(fail, 0, -3);  // non-finite Ritz value: breakdown
  int rank = 0;
  for (int j = 0; j < p; ++j) {
    double lj = H[idx2(j, j, ldh)];
    rank += rank_before((double)lj, j, (double)li, i);
  }
  ord[rank] = i;
}

// Usel[:, j] = U[:, ord[p-keep+j]], theta[j] = H[ord, ord]; npos into *npos
__global__ void k_select_top(const double* H, int ldh, const double* U, int ldu, int p, int keep, const int* ord,
                             double* Usel, double* theta, int* npos) {
  int j = blockIdx.x;
  if (j >= keep) return;
  int col = ord[p - keep + j];
  for (int i = threadIdx.x; i < p; i += blockDim.x) Usel[idx2(i, j, p)] = U[idx2(i, col, ldu)];
  if (threadIdx.x == 0) theta[j] = H[idx2(col, col, ldh)];
  if (j == 0 && threadIdx.x == 0) {
    int c = 0;
    for (int q = 0; q < p; ++q) c += H[idx2(q, q, ldh)] > 0.0;
    *npos = c;
  }
}

// Copy the outcome of a large Rayleigh-Ritz step into the control block.
__global__ void k_rr_large_finish(Ctl* ctl, const GridBar* b) {
  if (threadIdx.x == 0) {
    ctl->rr_fail = b->fail ? b->fail : (b->err ? -1 : 0);
    ctl->sweeps += b->sweeps;
  }
}

template __global__ void k_chol_inv_coop<double>(double*, double*, int, double, GridBar*);
template __global__ void k_chol_inv_coop<float>(double*, double*, int, double, GridBar*);
template __global__ void k_jacobi_coop<double>(double*, double*, int, double*, int, int, double, double, int,
                                               const double*, GridBar*);
template __global__ void k_jacobi_coop<float>(double*, double*, int, double*, int, int, double, double, int,
                                              const double*, GridBar*);

}  // namespace sdpg
