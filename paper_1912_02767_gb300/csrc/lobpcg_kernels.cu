// lobpcg_kernels.cu -- CUDA-core kernels of the projection onto the PSD cone:
// batched block products (W times a block, Gram matrices, block updates and
// the rank-k reconstruction of Eq. 2), the per-instance Rayleigh-Ritz step
// (Algorithm 2: Cholesky QR + symmetric eigendecomposition by parallel
// cyclic Jacobi) and the residual/normalisation kernels of Algorithm 3.
//
// Products run in `TC` arithmetic (double for the FP64 path, float for the
// mixed path's Grams and updates); storage is FP64 throughout.
#include "common.cuh"
#include "kernels.h"

namespace sdpg {

// ---------------------------------------------------------------------------
// Batched tiled GEMM: C = alpha op(A) op(B) (+ beta C), 64x64 tiles, k-step
// 16, 256 threads with a 4x4 register tile each.  op(A) is M x K, op(B) is
// K x N; TA: A stored K x M (column-major), TB: B stored N x K.
// Job `j` covers tiles_m * tiles_n * splits CTAs; split s handles a K-range
// and (EPI_PARTIAL) writes its own partial matrix at C + s*ldc*N.
// ---------------------------------------------------------------------------
template <bool TA, bool TB, typename TC>
__global__ void __launch_bounds__(256) k_gemm(const GemmJob* jobs, WorkMap wm) {
  __shared__ TC As[16][65];
  __shared__ TC Bs[16][65];
  int local;
  const int ji = find_inst(wm, blockIdx.x, &local);
  const GemmJob J = jobs[ji];
  const int tiles_mn = J.tiles_m * J.tiles_n;
  const int split = local / tiles_mn;
  const int t = local - split * tiles_mn;
  const int r0 = (t % J.tiles_m) * 64, c0 = (t / J.tiles_m) * 64;
  int kchunk = (J.K + J.splits - 1) / J.splits;
  kchunk = (kchunk + 15) & ~15;
  const int k0 = split * kchunk;
  const int k1 = min(J.K, k0 + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  TC acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (TC)0;
  for (int kk = k0; kk < k1; kk += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lin = tid + e * 256, i, k;
      if (!TA) { i = lin & 63; k = lin >> 6; }
      else { k = lin & 15; i = lin >> 4; }
      int gi = r0 + i, gk = kk + k;
      TC val = (TC)0;
      if (gi < J.M && gk < k1) {
        double a = TA ? J.A[(size_t)gk + (size_t)gi * J.lda] : J.A[(size_t)gi + (size_t)gk * J.lda];
        if (J.colscale) a *= J.colscale[gk];
        val = (TC)a;
      }
      As[k][i] = val;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lin = tid + e * 256, j, k;
      if (!TB) { k = lin & 15; j = lin >> 4; }
      else { j = lin & 63; k = lin >> 6; }
      int gj = c0 + j, gk = kk + k;
      TC val = (TC)0;
      if (gj < J.N && gk < k1)
        val = (TC)(TB ? J.B[(size_t)gj + (size_t)gk * J.ldb] : J.B[(size_t)gk + (size_t)gj * J.ldb]);
      Bs[k][j] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      TC a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[k][tx + 16 * q]; b[q] = Bs[k][ty + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] += a[q] * b[r];
    }
    __syncthreads();
  }
  // epilogue: thread (tx, ty) owns rows r0 + tx + 16q, cols c0 + ty + 16r
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int j = c0 + ty + 16 * r;
    if (j >= J.N) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int i = r0 + tx + 16 * q;
      if (i >= J.M) continue;
      double v = (double)acc[q][r];
      size_t o = (size_t)i + (size_t)j * J.ldc;
      if (J.epi == EPI_PARTIAL) {
        J.C[o + (size_t)split * J.ldc * J.N] = v;
      } else if (J.epi == EPI_STORE) {
        J.C[o] = J.beta == 0.0 ? J.alpha * v : J.alpha * v + J.beta * J.C[o];
      } else {  // EPI_RECON_POS / EPI_RECON_NEG: Z = [W] + acc, Y = rho (W - Z)
        double w = J.Eb[o];
        double z = (J.epi == EPI_RECON_NEG ? w : 0.0) + v;
        J.C[o] = z;
        J.C2[o] = J.rho * (w - z);
      }
    }
  }
}

// Sum the split-K partials of a Gram job; optionally symmetrise.
__global__ void k_gram_reduce(const GemmJob* jobs, WorkMap wm, int symmetrize) {
  int local;
  const int ji = find_inst(wm, blockIdx.x, &local);
  const GemmJob J = jobs[ji];
  int e = local * blockDim.x + threadIdx.x;
  if (e >= J.M * J.N) return;
  int i = e % J.M, j = e / J.M;
  double s = 0.0, st = 0.0;
  size_t stride = (size_t)J.ldc * J.N;
  for (int k = 0; k < J.splits; ++k) {
    s += J.C[(size_t)i + (size_t)j * J.ldc + k * stride];
    if (symmetrize) st += J.C[(size_t)j + (size_t)i * J.ldc + k * stride];
  }
  J.C2[(size_t)i + (size_t)j * J.M] = symmetrize ? 0.5 * (s + st) : s;
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi on one CTA (round-robin pairs, thresholds of RRConst<T>):
// the eigensolver of the allocation-free projection below.  Rayleigh-Ritz
// (Algorithm 2) itself is k_rr_smem (Jacobi comparator) in this file and
// k_rr_tri / rr_wide (tridiagonal route) in rr_tri.cu / rr_wide.cu.
// ---------------------------------------------------------------------------
template <typename T>
struct RRConst;
template <>
struct RRConst<double> {
  static constexpr double jac_rel = kJacobiRel64, jac_abs = kJacobiAbs64;
  static constexpr double piv_min = 1e-12;
  static constexpr int max_sweeps = 40;
};
template <>
struct RRConst<float> {
  static constexpr double jac_rel = kJacobiRel32, jac_abs = kJacobiAbs32;
  static constexpr double piv_min = 1e-6;
  static constexpr int max_sweeps = 25;
};

// round-robin (circle method) pairing for np (even) indices, round r, pair k
__device__ __forceinline__ void rr_pair(int r, int k, int np, int* a, int* b) {
  if (k == 0) {
    *a = 0;
    *b = 1 + (r % (np - 1));
  } else {
    *a = 1 + (r + k) % (np - 1);
    *b = 1 + (r - k + (np - 1)) % (np - 1);
  }
}

// CTA-wide cyclic Jacobi (parallel ordering) on symmetric H (p x p, ld ldh),
// accumulating the rotations into U (set to I here).  Returns sweeps.
template <typename T>
__device__ int cta_jacobi(int p, double* H, int ldh, double* U, int ldu, double* shc, double* shs, int* sha,
                          int* shb, double* red) {
  const int np = p + (p & 1), P2 = np / 2;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) U[idx2(t % p, t / p, ldu)] = (t % p == t / p) ? 1.0 : 0.0;
  // ||H||_F
  double part = 0.0;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    double h = H[idx2(t % p, t / p, ldh)];
    part += h * h;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  __shared__ double thr;
  __shared__ int rotated;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    thr = RRConst<T>::jac_abs * sqrt(s) / (double)(p > 0 ? p : 1);
  }
  __syncthreads();
  int sweep = 0;
  if (p < 2) return 0;
  for (; sweep < RRConst<T>::max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = threadIdx.x; k < P2; k += blockDim.x) {
        int a, b;
        rr_pair(r, k, np, &a, &b);
        double c = 1.0, s = 0.0;
        if (a < p && b < p) {
          T hab = (T)H[idx2(a, b, ldh)];
          T haa = (T)H[idx2(a, a, ldh)], hbb = (T)H[idx2(b, b, ldh)];
          if (jacobi_rotates((double)hab, (double)haa, (double)hbb, RRConst<T>::jac_rel, thr)) {
            T tau = (hbb - haa) / ((T)2 * hab);
            T tt = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
            T cc = (T)1 / sqrt((T)1 + tt * tt);
            c = (double)cc;
            s = (double)(tt * cc);
            rotated = 1;
          }
        }
        shc[k] = c; shs[k] = s; sha[k] = a; shb[k] = b;
      }
      __syncthreads();
      // two-sided update of every 2x2 block (pair i rows, pair j cols)
      for (int e = threadIdx.x; e < P2 * P2; e += blockDim.x) {
        int ki = e % P2, kj = e / P2;
        int ai = sha[ki], bi = shb[ki], aj = sha[kj], bj = shb[kj];
        T ci = (T)shc[ki], si = (T)shs[ki], cj = (T)shc[kj], sj = (T)shs[kj];
        bool vai = ai < p, vbi = bi < p, vaj = aj < p, vbj = bj < p;
        T haa = (vai && vaj) ? (T)H[idx2(ai, aj, ldh)] : (T)0;
        T hab = (vai && vbj) ? (T)H[idx2(ai, bj, ldh)] : (T)0;
        T hba = (vbi && vaj) ? (T)H[idx2(bi, aj, ldh)] : (T)0;
        T hbb = (vbi && vbj) ? (T)H[idx2(bi, bj, ldh)] : (T)0;
        T taa = cj * haa - sj * hab, tab = sj * haa + cj * hab;
        T tba = cj * hba - sj * hbb, tbb = sj * hba + cj * hbb;
        T naa = ci * taa - si * tba, nba = si * taa + ci * tba;
        T nab = ci * tab - si * tbb, nbb = si * tab + ci * tbb;
        if (ki == kj && si != (T)0) { nab = (T)0; nba = (T)0; }
        if (vai && vaj) H[idx2(ai, aj, ldh)] = (double)naa;
        if (vai && vbj) H[idx2(ai, bj, ldh)] = (double)nab;
        if (vbi && vaj) H[idx2(bi, aj, ldh)] = (double)nba;
        if (vbi && vbj) H[idx2(bi, bj, ldh)] = (double)nbb;
      }
      for (int e = threadIdx.x; e < p * P2; e += blockDim.x) {
        int row = e % p, k = e / p;
        int a = sha[k], b = shb[k];
        if (a >= p || b >= p || shs[k] == 0.0) continue;
        T c = (T)shc[k], s = (T)shs[k];
        T ua = (T)U[idx2(row, a, ldu)], ub = (T)U[idx2(row, b, ldu)];
        U[idx2(row, a, ldu)] = (double)(c * ua - s * ub);
        U[idx2(row, b, ldu)] = (double)(s * ua + c * ub);
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  return sweep + 1;
}


// ---------------------------------------------------------------------------
// Residuals of Algorithm 3: R = A X - X Theta (fresh columns: Theta = 0)
// written to the spare buffer S[1-par] at columns [m, 2m); Delta X and
// A Delta X copied to S[1-par] / AS[1-par] at [2m, 2m+mP); column norms in
// resn.  grid: (instance, column) over columns [0, m + mP)
// ---------------------------------------------------------------------------
__global__ void k_resid(Inst* insts, WorkMap wm) {
  __shared__ double sh[32];
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const Ctl* ctl = I.ctl;
  const int m = ctl->m, mP = ctl->mP, n = I.n, ld = I.ld;
  const int j = local;
  if (j >= m + mP) return;
  const double* S = I.S[I.par];
  const double* AS = I.AS[I.par];
  double* T = I.S[1 - I.par];
  double* AT = I.AS[1 - I.par];
  double part = 0.0;
  if (j < m) {
    double th = (j < m - ctl->nfresh) ? I.theta[j] : 0.0;
    const double* x = S + (size_t)j * ld;
    const double* ax = AS + (size_t)j * ld;
    double* r = T + (size_t)(m + j) * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double v = ax[i] - th * x[i];
      r[i] = v;
      part += v * v;
    }
  } else {
    size_t off = (size_t)(2 * m + (j - m)) * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double v = S[off + i];
      T[off + i] = v;
      AT[off + i] = AS[off + i];
      part += v * v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    I.resn[j] = sqrt(s);
  }
}

// Per instance: convergence test (every Ritz pair of the block within tol,
// no fresh columns), residual summaries, and the columns whose R and
// Delta X enter the next trial subspace [X, R_act, dX_act]: every column
// with a nonzero residual (Algorithm 3), or with soft locking only those
// still above tol (fresh columns always).
// last_allowed = 0: the step budget is spent, stop.
__global__ void k_resid_finish(Inst* insts, const int* list, int last_allowed) {
  const Inst& I = insts[list[blockIdx.x]];
  Ctl* c = I.ctl;
  if (threadIdx.x != 0) return;
  const int m = c->m, mP = c->mP;
  double rmax = 0.0, rpos2 = 0.0, thmin = 1e300;
  int npos = 0, ma = 0, mPa = 0;
  for (int j = 0; j < m; ++j) {
    double r = I.resn[j];
    bool fresh = j >= m - c->nfresh;
    rmax = fmax(rmax, r);
    if (!fresh) thmin = fmin(thmin, fabs(I.theta[j]));
    if (!fresh && I.theta[j] > 0.0) {
      ++npos;
      rpos2 += r * r;
    }
    bool act = fresh || !c->soft_lock || r > c->tol;  // Algorithm 3: every residual (soft locking: the unconverged)
    I.slot[j] = act && r > 0.0 ? ma++ : -1;
  }
  for (int j = 0; j < mP; ++j)
    if (I.slot[j] >= 0 && I.resn[m + j] > 0.0) ++mPa;
  c->res_max = rmax;
  c->res_pos2 = rpos2;
  c->thmin = thmin;
  c->npos = npos;
  c->ma = ma;
  c->mPa = mPa;
  bool conv = (c->nfresh == 0) && (rmax <= c->tol);
  if (conv || !last_allowed || ma == 0) c->active = 0;
  c->p = m + ma + mPa;
  c->keep = m;
}

// Compact the active residual and Delta X columns into S[par] after X,
// scaled to unit norm (the trial subspace is unchanged by column scaling;
// Cholesky QR sees a well-scaled Gram matrix).  Reads only the spare
// buffers written by k_resid.  grid: (instance, column) over [0, m + mP).
__global__ void k_compact(Inst* insts, WorkMap wm) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const Ctl* ctl = I.ctl;
  const int m = ctl->m, mP = ctl->mP, ma = ctl->ma;
  const int j = local;
  if (!ctl->active || j >= m + mP) return;
  const int jj = j < m ? j : j - m;
  int sl = I.slot[jj];
  if (sl < 0) return;
  double* S = I.S[I.par];
  double* AS = I.AS[I.par];
  const double* T = I.S[1 - I.par];
  const double* AT = I.AS[1 - I.par];
  if (j < m) {
    double sc = 1.0 / I.resn[j];
    const double* src = T + (size_t)(m + j) * I.ld;
    double* dst = S + (size_t)(m + sl) * I.ld;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) dst[i] = sc * src[i];
  } else {
    double nr = I.resn[m + jj];
    if (!(nr > 0.0)) return;
    // rank of this Delta X column among the active ones
    int r = 0;
    for (int q = 0; q < jj; ++q) r += (I.slot[q] >= 0 && I.resn[m + q] > 0.0);
    double sc = 1.0 / nr;
    size_t so = (size_t)(2 * m + jj) * I.ld, dof = (size_t)(m + ma + r) * I.ld;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
      S[dof + i] = sc * T[so + i];
      AS[dof + i] = sc * AT[so + i];
    }
  }
}

// Fresh Gaussian columns of the expansion (the expansion step of Algorithm 3), from
// the same Philox stream as the oracle: (row, col, draw, stream) with
// draw = expansion count and stream = ADMM iteration.
__global__ void k_fill_random(Inst* insts, WorkMap wm, const int* col0, const int* ncols, const int* draw,
                              const unsigned* stream, unsigned long long seed) {
  int local;
  const int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const int j = local;
  if (j >= ncols[ii]) return;
  double* S = I.S[I.par];
  double* dst = S + (size_t)(col0[ii] + j) * I.ld;
  for (int i = threadIdx.x; i < I.n; i += blockDim.x)
    dst[i] = philox_normal(seed, stream[ii], (uint32_t)draw[ii], (uint32_t)i, (uint32_t)j);
}

// Explicit instantiations
template __global__ void k_gemm<false, false, double>(const GemmJob*, WorkMap);
template __global__ void k_gemm<true, false, double>(const GemmJob*, WorkMap);
template __global__ void k_gemm<false, true, double>(const GemmJob*, WorkMap);
template __global__ void k_gemm<false, false, float>(const GemmJob*, WorkMap);
template __global__ void k_gemm<true, false, float>(const GemmJob*, WorkMap);
template __global__ void k_gemm<false, true, float>(const GemmJob*, WorkMap);

}  // namespace sdpg

// ---------------------------------------------------------------------------
// Projection of a small matrix without any device allocation.
//
// For callers that cannot allocate device memory: code that runs while a
// CUDA stream is being captured into a graph (cudaMalloc is not allowed
// there), or applications whose memory is fully pooled up front and which
// forbid allocation after start-up.  The scratch lives in one file-scope
// __device__ array that every GPU loading this library holds until exit.
// It is shared by all calls: calls that overlap on the GPU (two streams,
// two host threads) race on it, so the caller must serialise them.  Each
// call overwrites every scratch element it reads, so no state carries over.
//
// It is the Rayleigh-Ritz kernel specialised to the trial subspace S = I:
// G = I needs no Cholesky, and the eigendecomposition of M = W by the
// CTA-wide Jacobi gives Pi(W) = sum over lambda_k > 0 of lambda_k u_k u_k^T.
// ---------------------------------------------------------------------------
#include "../../include/sdpgpu.h"

namespace sdpg {
static __device__ __align__(256) double g_noalloc_scratch[2 * SDP_NOALLOC_MAX_N * SDP_NOALLOC_MAX_N];

__global__ void __launch_bounds__(1024) k_project_small_noalloc(int n, const double* W, double* out, double* scratch) {
  __shared__ double shc[SDP_NOALLOC_MAX_N / 2 + 1], shs[SDP_NOALLOC_MAX_N / 2 + 1];
  __shared__ int sha[SDP_NOALLOC_MAX_N / 2 + 1], shb[SDP_NOALLOC_MAX_N / 2 + 1];
  __shared__ double red[32];
  double* H = scratch;
  double* U = scratch + (size_t)n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t % n, j = t / n;
    H[t] = 0.5 * (W[i + (size_t)j * n] + W[j + (size_t)i * n]);
  }
  __syncthreads();
  cta_jacobi<double>(n, H, n, U, n, shc, shs, sha, shb, red);
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t % n, j = t / n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
      double l = H[k + (size_t)k * n];
      if (l > 0.0) acc += l * U[i + (size_t)k * n] * U[j + (size_t)k * n];
    }
    out[t] = acc;
  }
}
}  // namespace sdpg

extern "C" int sdp_project_psd_noalloc(int n, const double* W, double* out, void* cuda_stream) {
  if (n < 1 || n > SDP_NOALLOC_MAX_N || !W || !out) return SDP_E_INVALID;
  // host code must not use the array's name as a device address: ask the
  // runtime for the current device's address of the array on every call
  // (cheap after the first call on a device, which may load the module; a
  // per-process cache would go stale after a device reset)
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, sdpg::g_noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();  // consume this call's own error
    return SDP_E_CUDA;
  }
  // the launch's own status (an error left pending by earlier, unrelated
  // work is neither reported nor cleared here)
  double* sp = (double*)scratch;
  void* args[] = {(void*)&n, (void*)&W, (void*)&out, (void*)&sp};
  const cudaError_t e = cudaLaunchKernel((const void*)sdpg::k_project_small_noalloc, dim3(1), dim3(1024), args, 0,
                                         (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SDP_E_CUDA;
  }
  return SDP_OK;
}


namespace sdpg {
// ---------------------------------------------------------------------------
// Rayleigh-Ritz (Algorithm 2) with Cholesky-QR orthonormalisation
// (Q = S L^{-T}, never formed), one CTA per instance, by cyclic Jacobi: the
// comparator of the tridiagonal route (rr_method = 1).  Cholesky of G,
// L^{-1}, H = L^{-1} M L^{-T}, parallel cyclic Jacobi, sort,
// Coef = L^{-T} U_top; the matrices stay in shared memory (mode 0: both,
// mode 1: one) or in the instance's global scratch (mode 2).
// ---------------------------------------------------------------------------
// Dynamic shared memory: [A: p*p T][B: p*p T] (as the mode keeps them)
// followed by the per-round rotation table and the sort order
// (rr_table_bytes in kernels.h).
template <typename T>
__global__ void __launch_bounds__(1024) k_rr_smem(Inst* insts, const int* list, int u_global, int p_launch) {
  const Inst& I = insts[list[blockIdx.x]];
  Ctl* ctl = I.ctl;
  const int p = ctl->p, keep = ctl->keep;
  if (p < 1 || p > p_launch || p > kRRGlobalMax || keep < 1 || keep > p) {  // launch sized for another width: refuse, no access
    if (threadIdx.x == 0) ctl->rr_fail = -2;
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  // the two p x p workspaces (A: G -> L -> H, B: L^{-1} -> U): both in
  // shared memory (u_global = 0), B in the instance's global scratch
  // (u_global = 1), or both there (u_global = 2); global scratch stays
  // L2-resident
  const int in_smem = u_global == 0 ? 2 : u_global == 1 ? 1 : 0;
  T* A = u_global == 2 ? (T*)I.gpart : (T*)smraw;
  T* B = u_global ? (T*)I.U : A + p * p;
  unsigned char* tab = smraw + (size_t)in_smem * p * p * sizeof(T);
  const int P2max = (p + 1) / 2;
  T* cs0 = (T*)tab;
  T* cs1 = cs0 + P2max;
  int* pa = (int*)(cs1 + P2max);
  int* pb = pa + P2max;
  int* ord = pb + P2max;
  __shared__ int fail, rotated;
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = p + (p & 1), P2 = np / 2;
  // 1. A = G, Cholesky in place (lower)
  for (int t = tid; t < p * p; t += nt) A[t] = (T)I.G[t];
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (tid == 0) {
      T d = A[j + j * p];
      if (!(d > (T)(I.piv_loose ? 1e-6 : RRConst<T>::piv_min))) fail = j + 1;
      A[j + j * p] = sqrt(d > (T)0 ? d : (T)1);
    }
    __syncthreads();
    if (fail) break;
    T ljj = A[j + j * p];
    for (int i = j + 1 + tid; i < p; i += nt) A[i + j * p] /= ljj;
    __syncthreads();
    int w = p - j - 1;
    for (int t = tid; t < w * w; t += nt) {
      int r = t % w, c = t / w;
      if (r < c) continue;
      A[(j + 1 + r) + (j + 1 + c) * p] -= A[(j + 1 + r) + j * p] * A[(j + 1 + c) + j * p];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) ctl->rr_fail = fail;
    return;
  }
  // 2. B = L^{-1}: column c by one thread (p <= 160 threads busy)
  for (int c = tid; c < p; c += nt) {
    for (int i = 0; i < c; ++i) B[i + c * p] = (T)0;
    for (int i = c; i < p; ++i) {
      T acc = (i == c) ? (T)1 : (T)0;
      for (int k = c; k < i; ++k) acc -= A[i + k * p] * B[k + c * p];
      B[i + c * p] = acc / A[i + i * p];
    }
  }
  __syncthreads();
  // keep L^{-1} in global for the coefficients; T1 = Linv M -> global scratch
  for (int t = tid; t < p * p; t += nt) I.Linv[t] = (double)B[t];
  for (int t = tid; t < p * p; t += nt) {
    int i = t % p, j = t / p;
    T acc = 0;
    for (int k = 0; k <= i; ++k) acc += B[i + k * p] * (T)I.M[k + j * p];
    I.H[t] = (double)acc;
  }
  __syncthreads();
  // 3. A = H = T1 Linv^T (symmetric: lower computed, mirrored)
  for (int t = tid; t < p * p; t += nt) {
    int i = t % p, j = t / p;
    if (i < j) continue;
    T acc = 0;
    for (int k = 0; k <= j; ++k) acc += (T)I.H[i + k * p] * B[j + k * p];
    A[i + j * p] = acc;
    A[j + i * p] = acc;
  }
  __syncthreads();
  // 4. Jacobi on A, rotations accumulated in B (= U)
  for (int t = tid; t < p * p; t += nt) B[t] = (t % p == t / p) ? (T)1 : (T)0;
  double part = 0.0;
  for (int t = tid; t < p * p; t += nt) part += (double)A[t] * (double)A[t];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  __shared__ double thr;
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) s += red[w];
    thr = RRConst<T>::jac_abs * sqrt(s) / (double)p;
  }
  __syncthreads();
  int sweeps = 0;
  for (int sweep = 0; sweep < RRConst<T>::max_sweeps && p >= 2; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = tid; k < P2; k += nt) {
        int a, b;
        rr_pair(r, k, np, &a, &b);
        T c = (T)1, s = (T)0;
        if (a < p && b < p) {
          T hab = A[a + b * p];
          T haa = A[a + a * p], hbb = A[b + b * p];
          if (jacobi_rotates((double)hab, (double)haa, (double)hbb, RRConst<T>::jac_rel, thr)) {
            T tau = (hbb - haa) / ((T)2 * hab);
            T tt = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
            c = (T)1 / sqrt((T)1 + tt * tt);
            s = tt * c;
            rotated = 1;
          }
        }
        cs0[k] = c; cs1[k] = s; pa[k] = a; pb[k] = b;
      }
      __syncthreads();
      for (int e = tid; e < P2 * P2; e += nt) {
        int ki = e % P2, kj = e / P2;
        T si = cs1[ki], sj = cs1[kj];
        if (si == (T)0 && sj == (T)0) continue;
        int ai = pa[ki], bi = pb[ki], aj = pa[kj], bj = pb[kj];
        T ci = cs0[ki], cj = cs0[kj];
        bool vai = ai < p, vbi = bi < p, vaj = aj < p, vbj = bj < p;
        T haa = (vai && vaj) ? A[ai + aj * p] : (T)0;
        T hab = (vai && vbj) ? A[ai + bj * p] : (T)0;
        T hba = (vbi && vaj) ? A[bi + aj * p] : (T)0;
        T hbb = (vbi && vbj) ? A[bi + bj * p] : (T)0;
        T taa = cj * haa - sj * hab, tab = sj * haa + cj * hab;
        T tba = cj * hba - sj * hbb, tbb = sj * hba + cj * hbb;
        T naa = ci * taa - si * tba, nba = si * taa + ci * tba;
        T nab = ci * tab - si * tbb, nbb = si * tab + ci * tbb;
        if (ki == kj && si != (T)0) { nab = (T)0; nba = (T)0; }
        if (vai && vaj) A[ai + aj * p] = naa;
        if (vai && vbj) A[ai + bj * p] = nab;
        if (vbi && vaj) A[bi + aj * p] = nba;
        if (vbi && vbj) A[bi + bj * p] = nbb;
      }
      for (int e = tid; e < p * P2; e += nt) {
        int row = e % p, k = e / p;
        T s = cs1[k];
        if (s == (T)0) continue;
        int a = pa[k], b = pb[k];
        if (a >= p || b >= p) continue;
        T c = cs0[k];
        T ua = B[row + a * p], ub = B[row + b * p];
        B[row + a * p] = c * ua - s * ub;
        B[row + b * p] = s * ua + c * ub;
      }
      __syncthreads();
    }
    ++sweeps;
    if (!rotated) break;
    __syncthreads();
  }
  // 5. ascending order
  for (int i = tid; i < p; i += nt) {
    T li = A[i + i * p];
    int rank = 0;
    for (int j = 0; j < p; ++j) {
      T lj = A[j + j * p];
      rank += rank_before((double)lj, j, (double)li, i);
    }
    ord[rank] = i;
  }
  __syncthreads();
  // 6. Coef = Linv^T U[:, top keep]
  for (int t = tid; t < p * keep; t += nt) {
    int i = t % p, j = t / p;
    int col = ord[p - keep + j];
    T acc = 0;
    for (int k = i; k < p; ++k) acc += (T)I.Linv[k + i * p] * B[k + col * p];
    I.Coef[i + j * p] = (double)acc;
  }
  for (int j = tid; j < keep; j += nt) I.theta[j] = (double)A[ord[p - keep + j] * (p + 1)];
  if (tid == 0) {
    int c = 0, bad = 0;
    for (int j = 0; j < p; ++j) {
      c += A[j + j * p] > (T)0;
      bad |= !isfinite((double)A[j + j * p]);
    }
    ctl->npos_rr = c;
    ctl->rr_fail = bad ? -3 : 0;  // non-finite Ritz values: breakdown
    ctl->sweeps += sweeps;
  }
}

template __global__ void k_rr_smem<double>(Inst*, const int*, int, int);
template __global__ void k_rr_smem<float>(Inst*, const int*, int, int);
}  // namespace sdpg
