// bj_eig.cu -- two-sided block Jacobi eigendecomposition of a symmetric
// p x p matrix H (the Rayleigh-Ritz matrix of Algorithm 2 / 3 for wide
// trial subspaces).  Indices are split into blocks of BJ_B; a sweep pairs
// every two blocks once (round-robin tournament over blocks).  In a round
// each pair (I, J) diagonalises its (|I|+|J|)-square submatrix in shared
// memory with the CTA-wide cyclic Jacobi (one CTA per pair) and the
// resulting orthogonal Q is applied to the block rows, then the block
// columns of H, and to the block columns of U.  A sweep is p / BJ_B
// rounds instead of the p rounds of scalar Jacobi.  Convergence: the
// off-diagonal Frobenius norm of the sweep's subproblems below eps ||H||_F.
#include "common.cuh"
#include "kernels.h"

namespace sdpg {

static constexpr int BJ_B = 32;            // block size
static constexpr int BJ_S = 2 * BJ_B;      // subproblem size

__device__ __forceinline__ void bj_pair(int r, int k, int np, int* a, int* b) {
  if (k == 0) {
    *a = 0;
    *b = 1 + (r % (np - 1));
  } else {
    *a = 1 + (r + k) % (np - 1);
    *b = 1 + (r - k + (np - 1)) % (np - 1);
  }
}

// global index of local position q (0..sz-1) of pair blocks (I, J)
__device__ __forceinline__ int bj_index(int q, int I, int sI, int J) {
  return q < sI ? I * BJ_B + q : J * BJ_B + (q - sI);
}
__device__ __forceinline__ int bj_bsize(int I, int nb, int p) {
  if (I >= nb) return 0;
  return min(BJ_B, p - I * BJ_B);
}

// One CTA per pair: load the submatrix, record its off-diagonal mass,
// diagonalise it, store Q (BJ_S x BJ_S, column-major) for the pair.
template <typename T>
__global__ void __launch_bounds__(512) k_bj_sub(const double* H, int ldh, int p, int round, double* Q, double* offp) {
  __shared__ T S[BJ_S][BJ_S + 1];
  __shared__ T V[BJ_S][BJ_S + 1];
  __shared__ T cs[2][BJ_S / 2];
  __shared__ int pa[BJ_S / 2], pb[BJ_S / 2];
  __shared__ double red[16];
  __shared__ int rotated;
  const int nb = (p + BJ_B - 1) / BJ_B, np = nb + (nb & 1);
  const int k = blockIdx.x;
  int I, J;
  bj_pair(round, k, np, &I, &J);
  const int sI = bj_bsize(I, nb, p), sJ = bj_bsize(J, nb, p);
  const int sz = sI + sJ;
  const int tid = threadIdx.x, nt = blockDim.x;
  double off = 0.0, all = 0.0;
  for (int t = tid; t < BJ_S * BJ_S; t += nt) {
    int i = t % BJ_S, j = t / BJ_S;
    T v = (T)0;
    if (i < sz && j < sz) {
      v = (T)H[idx2(bj_index(i, I, sI, J), bj_index(j, I, sI, J), ldh)];
      if (i != j) off += (double)v * (double)v;
      all += (double)v * (double)v;
    }
    S[i][j] = v;
    V[i][j] = (i == j) ? (T)1 : (T)0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_down_sync(0xffffffffu, off, o);
    all += __shfl_down_sync(0xffffffffu, all, o);
  }
  __shared__ double red2[16];
  __shared__ double sthr;
  if ((tid & 31) == 0) { red[tid >> 5] = off; red2[tid >> 5] = all; }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0, a = 0.0;
    for (int w = 0; w < nt / 32; ++w) { s += red[w]; a += red2[w]; }
    offp[k] = s;
    // rotate while a pair exceeds a small multiple of the rounding level of
    // the subproblem (below it, rotations only chase rounding noise)
    sthr = 16.0 * (sizeof(T) == 4 ? 6e-8 : 1.1e-16) * sqrt(a) / (double)(sz > 0 ? sz : 1);
  }
  __syncthreads();
  // cyclic Jacobi on the sz x sz block: two sweeps (relaxed block Jacobi:
  // the outer sweeps finish what the inner ones leave, at a fraction of the
  // cost of diagonalising every subproblem to rounding level)
  const int snp = sz + (sz & 1), P2 = snp / 2;
  for (int sweep = 0; sweep < 2 && sz >= 2; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < snp - 1; ++r) {
      for (int q = tid; q < P2; q += nt) {
        int a, b;
        bj_pair(r, q, snp, &a, &b);
        T c = (T)1, s = (T)0;
        if (a < sz && b < sz) {
          T hab = S[a][b], haa = S[a][a], hbb = S[b][b];
          if (fabs((double)hab) > sthr) {
            T tau = (hbb - haa) / ((T)2 * hab);
            T tt = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
            c = (T)1 / sqrt((T)1 + tt * tt);
            s = tt * c;
            rotated = 1;
          }
        }
        cs[0][q] = c;
        cs[1][q] = s;
        pa[q] = a;
        pb[q] = b;
      }
      __syncthreads();
      for (int e = tid; e < P2 * P2; e += nt) {
        int ki = e % P2, kj = e / P2;
        T si = cs[1][ki], sj = cs[1][kj];
        if (si == (T)0 && sj == (T)0) continue;
        int ai = pa[ki], bi = pb[ki], aj = pa[kj], bj = pb[kj];
        T ci = cs[0][ki], cj = cs[0][kj];
        T haa = S[ai][aj], hab = S[ai][bj], hba = S[bi][aj], hbb = S[bi][bj];
        T taa = cj * haa - sj * hab, tab = sj * haa + cj * hab;
        T tba = cj * hba - sj * hbb, tbb = sj * hba + cj * hbb;
        T naa = ci * taa - si * tba, nba = si * taa + ci * tba;
        T nab = ci * tab - si * tbb, nbb = si * tab + ci * tbb;
        if (ki == kj && si != (T)0) { nab = (T)0; nba = (T)0; }
        S[ai][aj] = naa; S[ai][bj] = nab; S[bi][aj] = nba; S[bi][bj] = nbb;
      }
      for (int e = tid; e < BJ_S * P2; e += nt) {
        int row = e % BJ_S, q = e / BJ_S;
        T s = cs[1][q];
        if (s == (T)0) continue;
        int a = pa[q], b = pb[q];
        T c = cs[0][q];
        T ua = V[row][a], ub = V[row][b];
        V[row][a] = c * ua - s * ub;
        V[row][b] = s * ua + c * ub;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  __syncthreads();
  double* Qk = Q + (size_t)k * BJ_S * BJ_S;
  for (int t = tid; t < BJ_S * BJ_S; t += nt) Qk[t] = (double)V[t % BJ_S][t / BJ_S];
}

// H[rows of pair k, column tile] <- Q_k^T H[rows, tile]  (rows disjoint
// across pairs, so the update is in place)
template <typename T>
__global__ void __launch_bounds__(256) k_bj_rows(double* H, int ldh, int p, int round, const double* Q) {
  __shared__ T Qs[BJ_S][BJ_S + 1];
  __shared__ T Ht[BJ_S][65];
  const int nb = (p + BJ_B - 1) / BJ_B, np = nb + (nb & 1);
  const int k = blockIdx.x, c0 = blockIdx.y * 64;
  int I, J;
  bj_pair(round, k, np, &I, &J);
  const int sI = bj_bsize(I, nb, p), sJ = bj_bsize(J, nb, p), sz = sI + sJ;
  if (sz == 0 || c0 >= p) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Qk = Q + (size_t)k * BJ_S * BJ_S;
  for (int t = tid; t < BJ_S * BJ_S; t += nt) Qs[t % BJ_S][t / BJ_S] = (T)Qk[t];
  const int w = min(64, p - c0);
  for (int t = tid; t < BJ_S * 64; t += nt) {
    int q = t % BJ_S, c = t / BJ_S;
    Ht[q][c] = (q < sz && c < w) ? (T)H[idx2(bj_index(q, I, sI, J), c0 + c, ldh)] : (T)0;
  }
  __syncthreads();
  for (int t = tid; t < sz * w; t += nt) {
    int i = t % sz, c = t / sz;
    T acc = 0;
    for (int j = 0; j < sz; ++j) acc += Qs[j][i] * Ht[j][c];
    H[idx2(bj_index(i, I, sI, J), c0 + c, ldh)] = (double)acc;
  }
}

// M[row tile, cols of pair k] <- M[row tile, cols] Q_k for M = H (z = 0)
// and M = U (z = 1)
template <typename T>
__global__ void __launch_bounds__(256) k_bj_cols(double* H, int ldh, double* U, int ldu, int p, int round,
                                                 const double* Q) {
  __shared__ T Qs[BJ_S][BJ_S + 1];
  __shared__ T Mt[64][BJ_S + 1];
  const int nb = (p + BJ_B - 1) / BJ_B, np = nb + (nb & 1);
  const int k = blockIdx.x, r0 = blockIdx.y * 64;
  double* M = blockIdx.z == 0 ? H : U;
  const int ld = blockIdx.z == 0 ? ldh : ldu;
  int I, J;
  bj_pair(round, k, np, &I, &J);
  const int sI = bj_bsize(I, nb, p), sJ = bj_bsize(J, nb, p), sz = sI + sJ;
  if (sz == 0 || r0 >= p) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Qk = Q + (size_t)k * BJ_S * BJ_S;
  for (int t = tid; t < BJ_S * BJ_S; t += nt) Qs[t % BJ_S][t / BJ_S] = (T)Qk[t];
  const int h = min(64, p - r0);
  for (int t = tid; t < 64 * BJ_S; t += nt) {
    int r = t % 64, q = t / 64;
    Mt[r][q] = (r < h && q < sz) ? (T)M[idx2(r0 + r, bj_index(q, I, sI, J), ld)] : (T)0;
  }
  __syncthreads();
  for (int t = tid; t < h * sz; t += nt) {
    int r = t % h, i = t / h;
    T acc = 0;
    for (int j = 0; j < sz; ++j) acc += Mt[r][j] * Qs[j][i];
    M[idx2(r0 + r, bj_index(i, I, sI, J), ld)] = (double)acc;
  }
}

__global__ void k_set_identity(double* U, int ld, int p) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)p * p) return;
  int i = (int)(t % p), j = (int)(t / p);
  U[idx2(i, j, ld)] = i == j ? 1.0 : 0.0;
}

// Host driver: block-Jacobi sweeps until the subproblems' off-diagonal
// mass is below (eps ||H||_F)^2 or max_sweeps.  Q (npairs * BJ_S^2) and
// offp (npairs) are device scratch; offh pinned host scratch (npairs).
// Returns the number of sweeps, or -1 on a CUDA error.
// FP32 arithmetic only (the FP64 path uses the cooperative scalar Jacobi:
// a 64 x 64 FP64 subproblem on one SM would be the bottleneck).
int block_jacobi(cudaStream_t s, double* H, int ldh, double* U, int ldu, int p, bool f32, double eps,
                 const double* fro2_dev, int max_sweeps, double* Q, double* offp, double* offh) {
  if (!f32) return -1;
  const int nb = (p + BJ_B - 1) / BJ_B, np = nb + (nb & 1), npairs = np / 2;
  const int tiles = (p + 63) / 64;
  k_set_identity<<<(unsigned)(((long)p * p + 255) / 256), 256, 0, s>>>(U, ldu, p);
  if (cudaMemcpyAsync(offh, fro2_dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  const double thr2 = eps * eps * offh[0];
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int r = 0; r < np - 1; ++r) {
      k_bj_sub<float><<<npairs, 512, 0, s>>>(H, ldh, p, r, Q, offp + (size_t)r * npairs);
      k_bj_rows<float><<<dim3(npairs, tiles), 256, 0, s>>>(H, ldh, p, r, Q);
      k_bj_cols<float><<<dim3(npairs, tiles, 2), 256, 0, s>>>(H, ldh, U, ldu, p, r, Q);
    }
    if (cudaMemcpyAsync(offh, offp, sizeof(double) * (size_t)(np - 1) * npairs, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    for (long q = 0; q < (long)(np - 1) * npairs; ++q) off += offh[q];
    // off counts each off-diagonal entry once per time its pair met; the
    // first sweep sees everything, later sweeps what fill-in left
    if (off <= thr2) {
      ++sweep;
      break;
    }
  }
  return cudaGetLastError() == cudaSuccess ? sweep : -1;
}

}  // namespace sdpg
