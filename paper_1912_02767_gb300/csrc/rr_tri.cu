// rr_tri.cu -- the Rayleigh-Ritz step of LOBPCG (Algorithm 3; Rayleigh-Ritz
// as in Algorithm 2) for one instance per CTA, by reduction to tridiagonal
// form.
//
// For the trial basis S (p columns) with Gram matrix G = S^T S and projected
// matrix M = S^T (W S) the step needs the top `keep` Ritz pairs of the pencil
// (M, G):
//   G = L~ D L~^T           (Cholesky-QR in LDL^T form, L~ unit lower)
//   H = D^{-1/2} L~^{-1} M L~^{-T} D^{-1/2}   (two unit-triangular solves)
//   H = Q T Q^T             (Householder tridiagonalization)
//   top `keep` eigenvalues of T by Sturm-sequence multisection (FP32, then
//   refined in FP64 by the division-free count of tri_common.cuh), their
//   eigenvectors by inverse iteration, orthonormalized within clusters of
//   close eigenvalues (classical Gram-Schmidt, twice), back-transformed by Q
//   Coef = L~^{-T} D^{-1/2} Y  (S Coef = the Ritz vectors)
// This is the textbook route for a few eigenpairs of a dense symmetric matrix
// (Householder reduction, Wilkinson's bisection on the Sturm count, inverse
// iteration); every phase is a short sequence of block-wide steps with one to
// four barriers each, instead of the p rounds per sweep of a parallel Jacobi
// method.
//
// Storage: H (p x p, odd leading dimension so that row and column walks are
// free of bank conflicts) and all vectors in shared memory; the Ritz block Y
// (p x keep) in shared memory too when it fits (`zsm`), else in the
// instance's global scratch U. L~ is kept in the scratch Linv and the
// inverse-iteration factors in gpart (both L2-resident).
#include "kernels.h"
#include "tri_common.cuh"

namespace sdpg {

using namespace tri;

template <typename T>
__global__ void __launch_bounds__(1024) k_rr_tri(Inst* insts, const int* list, int zsm, unsigned smem_launch) {
  const Inst& I = insts[list[blockIdx.x]];
  Ctl* ctl = I.ctl;
  const int p = ctl->p, keep = ctl->keep;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  // the launch must hold this width (refuse, touching nothing, otherwise)
  if (p < 1 || keep < 1 || keep > p || p > I.pcap || keep > I.mcap || (nt & 31) || nt > 1024 || p > nt ||
      rr_tri_smem_bytes(p, zsm ? keep : 0, (int)sizeof(T)) > smem_launch) {
    if (tid == 0) ctl->rr_fail = -2;
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ldp = p | 1;
  T* B = (T*)smraw;  // p x ldp: G -> LDL^T, then M -> H -> Householder vectors
  T* d = B + (size_t)p * ldp;
  T* e = d + p;
  T* e2 = e + p;
  T* tau = e2 + p;
  T* rs = tau + p;    // D^{-1/2}
  T* lam = rs + p;    // top eigenvalues of the scaled T, ascending
  T* sig = lam + p;   // inverse-iteration shifts
  T* vv = sig + p;    // Householder vector
  T* wv = vv + p;     // symv result / per-vector coefficients
  T* lcol = wv + p;   // 2 x p staging of one column (row) of L~
  T* part = lcol + 2 * p;  // 1024 partial sums
  T* Z = zsm ? part + 1024 : (T*)I.U;  // p x keep, row-major (i * keep + q)
  T* Lg = (T*)I.Linv;                  // L~, column-major, ld p
  T* WS = (T*)I.gpart;                 // inverse-iteration factors: 3 per row and vector
  __shared__ int s_fail, s_npos;
  __shared__ T s_red[32];
  __shared__ T s_sc[2];

  // breakdown threshold of Cholesky-QR: set by the precision the Gram was
  // formed in (FP32 Grams in the mixed modes), not by this kernel's type
  const T piv = I.piv_loose ? (T)1e-6 : (T)1e-12;  // the products' precision sets the breakdown threshold
  // ---- 1. G = L~ D L~^T (right-looking, lower triangle of B)
  for (int t = tid; t < p * p; t += nt) {
    const int i = t % p, j = t / p;
    if (i >= j) B[i + j * ldp] = (T)I.G[t];
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // pivot reciprocals (in `sig`, free until the shifts): each one computed
  // once, by the lane that finishes that pivot -- an FP64 division costs an
  // SM sub-partition about twelve FP64 issue slots, whatever the lanes
  T* rcp = sig;
  if (tid == 0) rcp[0] = (T)1 / B[0];
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const T djj = B[j + j * ldp];
    if (!(djj > piv)) {
      if (tid == 0) s_fail = j + 1;
      break;  // every thread reads the same pivot: uniform exit
    }
    const T inv = rcp[j];
    for (int c = j + 1 + wid; c < p; c += nw) {
      const T bc = B[c + j * ldp] * inv;
      for (int r = c + lane; r < p; r += 32) B[r + c * ldp] -= B[r + j * ldp] * bc;
      if (c == j + 1 && lane == 0) rcp[c] = (T)1 / B[c + c * ldp];  // the next pivot is final now
    }
    if (j > 0)  // column j-1 is no longer read: scale it to L~
      for (int r = j + tid; r < p; r += nt) B[r + (j - 1) * ldp] *= rcp[j - 1];
    __syncthreads();
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) ctl->rr_fail = s_fail;
    return;
  }
  for (int j = tid; j < p; j += nt) rs[j] = (T)1 / sqrt(B[j + j * ldp]);
  for (int t = tid; t < p * p; t += nt) {
    const int i = t % p, j = t / p;
    Lg[t] = i > j ? B[i + j * ldp] : (i == j ? (T)1 : (T)0);
  }
  __syncthreads();

  // ---- 2. B = L~^{-1} M L~^{-T} (unit lower solves from the left and the right)
  for (int t = tid; t < p * p; t += nt) {
    const int i = t % p, j = t / p;
    B[i + j * ldp] = (T)I.M[t];
  }
  for (int r = tid; r < p; r += nt) lcol[r] = Lg[r];
  __syncthreads();
  for (int j = 0; j + 1 < p; ++j) {  // rows below j -= L~[r, j] * row j
    const T* lc = lcol + (j & 1) * p;
    T* ln = lcol + ((j + 1) & 1) * p;
    for (int r = j + 1 + tid; r < p; r += nt) ln[r] = Lg[r + (size_t)(j + 1) * p];
    for (int c = wid; c < p; c += nw) {
      const T bj = B[j + c * ldp];
      for (int r = j + 1 + lane; r < p; r += 32) B[r + c * ldp] -= lc[r] * bj;
    }
    __syncthreads();
  }
  for (int r = tid; r < p; r += nt) lcol[r] = Lg[r];
  __syncthreads();
  for (int k = 0; k + 1 < p; ++k) {  // columns right of k -= L~[c, k] * column k
    const T* lc = lcol + (k & 1) * p;
    T* ln = lcol + ((k + 1) & 1) * p;
    for (int r = k + 1 + tid; r < p; r += nt) ln[r] = Lg[r + (size_t)(k + 1) * p];
    for (int c = k + 1 + wid; c < p; c += nw) {
      const T l = lc[c];
      for (int r = lane; r < p; r += 32) B[r + c * ldp] -= l * B[r + k * ldp];
    }
    __syncthreads();
  }
  // scale by D^{-1/2} on both sides and symmetrize
  for (int c = wid; c < p; c += nw)
    for (int r = c + lane; r < p; r += 32) {
      const T h = (T)0.5 * (B[r + c * ldp] + B[c + r * ldp]) * rs[r] * rs[c];
      B[r + c * ldp] = h;
      B[c + r * ldp] = h;
    }
  __syncthreads();

  // ---- 3. Householder tridiagonalization (full storage of the trailing block)
  for (int k = 0; k + 2 < p; ++k) {
    const int r = p - k - 1;  // the trailing block spans rows/columns k+1 .. p-1
    T* colk = B + (size_t)k * ldp + (k + 1);
    if (wid == 0) {
      T s = 0;
      for (int i = 1 + lane; i < r; i += 32) s += colk[i] * colk[i];
      s = warp_sum(s);
      const T x0 = colk[0];
      T beta = x0, t = 0, scale = 0;
      if (lane == 0 && s > (T)0) {  // P = I - t v v^T with v_0 = 1 maps x to beta e_1
        const T alpha = sqrt(x0 * x0 + s);
        beta = x0 >= (T)0 ? -alpha : alpha;
        t = (beta - x0) / beta;
        scale = (T)1 / (x0 - beta);
      }
      beta = __shfl_sync(0xffffffffu, beta, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      scale = __shfl_sync(0xffffffffu, scale, 0);
      for (int i = lane; i < r; i += 32) {
        const T v = i == 0 ? (T)1 : colk[i] * scale;
        vv[i] = v;
        if (i > 0) colk[i] = v;  // v kept below the subdiagonal for the back-transform
      }
      if (lane == 0) {
        d[k] = B[k + k * ldp];
        e[k] = beta;
        tau[k] = t;
      }
    }
    __syncthreads();
    const T t = tau[k];
    if (t == (T)0) continue;  // uniform: nothing to reflect
    const int R = (r + 31) & ~31;
    const int S = nt / R;
    {  // w = t A22 v: S column slices per row
      const int i = tid % R, s = tid / R;
      if (s < S && i < r) {
        const T* a = B + (size_t)(k + 1) * ldp + (k + 1) + i;
        T acc = 0;
        for (int c = s; c < r; c += S) acc += a[(size_t)c * ldp] * vv[c];
        part[s * R + i] = acc;
      }
    }
    __syncthreads();
    if (wid * 32 < r) {  // warps holding rows of w
      T pw = 0;
      if (tid < r) {
        T acc = 0;
        for (int s = 0; s < S; ++s) acc += part[s * R + tid];
        acc *= t;
        wv[tid] = acc;
        pw = acc * vv[tid];
      }
      pw = warp_sum(pw);
      if (lane == 0) s_red[wid] = pw;
    } else if (lane == 0) {
      s_red[wid] = (T)0;
    }
    __syncthreads();
    if (wid == 0) {  // K = t/2 w^T v, once
      T K = lane < nw ? s_red[lane] : (T)0;
      K = warp_sum(K) * ((T)0.5 * t);
      if (lane == 0) s_sc[0] = K;
    }
    __syncthreads();
    // A22 -= v w'^T + w' v^T with w' = w - K v
    if (wid < r) {
      const T K = s_sc[0];
      for (int c = wid; c < r; c += nw) {
        const T vc = vv[c], wc = wv[c] - K * vc;
        T* col = B + (size_t)(k + 1 + c) * ldp + (k + 1);
        for (int i = lane; i < r; i += 32) col[i] -= vv[i] * wc + (wv[i] - K * vv[i]) * vc;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (p >= 2) {
      d[p - 2] = B[(p - 2) + (p - 2) * ldp];
      d[p - 1] = B[(p - 1) + (p - 1) * ldp];
      e[p - 2] = B[(p - 1) + (p - 2) * ldp];
    } else {
      d[0] = B[0];
    }
  }
  __syncthreads();

  // ---- 4. scale T to unit norm (Gershgorin bound); non-finite data: breakdown
  if (wid == 0) {
    T lo = (T)0, hi = (T)0;
    bool bad = false;
    for (int i = lane; i < p; i += 32) {
      const T off = (i > 0 ? fabs(e[i - 1]) : (T)0) + (i + 1 < p ? fabs(e[i]) : (T)0);
      lo = fmin(lo, d[i] - off);
      hi = fmax(hi, d[i] + off);
      bad |= !isfinite(d[i]) || !isfinite(off);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      T nrm = fmax(fabs(lo), fabs(hi));
      nrm = nrm > (T)0 ? nrm : (T)1;
      s_sc[0] = nrm;
      s_sc[1] = (T)1 / nrm;
      if (bad) s_fail = -3;
    }
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) ctl->rr_fail = s_fail;
    return;
  }
  const T tn = s_sc[0], itn = s_sc[1];
  for (int i = tid; i < p; i += nt) {
    d[i] *= itn;
    if (i + 1 < p) {
      e[i] *= itn;
      e2[i] = e[i] * e[i];
    }
  }
  __syncthreads();

  // ---- 5. top `keep` eigenvalues: S-section on the Sturm count, one lane
  // group per eigenvalue, in FP32 (for T = double: to 64 ulps, then refined
  // in FP64 inside that bracket -- FP64 divisions are scarce, so the wide
  // search runs on the FP32 pipes)
  {
    float* d32 = (float*)vv;  // vv and wv are free until the back-transform
    float* e232 = (float*)wv;
    const bool dbl = sizeof(T) != sizeof(float);
    const float* db = dbl ? d32 : (const float*)d;
    const float* eb = dbl ? e232 : (const float*)e2;
    if (dbl) {
      for (int i = tid; i < p; i += nt) {
        d32[i] = (float)d[i];
        e232[i] = i + 1 < p ? (float)e2[i] : 0.0f;
      }
      __syncthreads();
    }
    int S2 = 32;
    while (S2 > 1 && S2 * keep > nt) S2 >>= 1;
    const float tol32 = (dbl ? 32.0f : 4.0f) * K<float>::eps;
    section_search<float>(db, eb, p, keep, S2, tid / S2, nt / S2, tol32, -1.01f, 1.01f, K<float>::safmin, lam,
                          false);
    if (dbl) {
      __syncthreads();
      // lanes per eigenvalue for the FP64 refinement (about 33 bits from
      // the FP32 bracket): every count is one FP64 chain, and warps sharing
      // an SM sub-partition share its FP64 issue, so take the S that needs
      // the fewest chains per sub-partition, ceil(warps / 4) * 33 / log2(S + 1)
      int S4 = 1;
      float best = 3.0e38f;
      for (int S = 1; S <= 32 && S * keep <= nt; S <<= 1) {
        const int W = (S * keep + 31) / 32;
        const float cost = (float)((W + 3) / 4) * (33.0f / log2f((float)S + 1.0f));
        if (cost < best * 0.999f) {
          best = cost;
          S4 = S;
        }
      }
      section_search<T>(d, e2, p, keep, S4, tid / S4, nt / S4, (T)4 * K<T>::eps, (T)(64.0f * K<float>::eps),
                        (T)0, (T)K<T>::safmin, lam, true);
    }
    if (tid == nt - 1) s_npos = p - sturm_below(d, e2, p, (T)0, (T)K<T>::safmin);
  }
  __syncthreads();
  if (tid == 0) {  // shifts at least 10 eps apart, so that equal eigenvalues get distinct vectors
    const T sep = (T)10 * K<T>::eps;
    T prev = lam[0];
    sig[0] = prev;
    for (int q = 1; q < keep; ++q) {
      T s = lam[q];
      if (s < prev + sep) s = prev + sep;
      sig[q] = s;
      prev = s;
    }
  }
  __syncthreads();

  // ---- 6. inverse iteration, one thread per eigenvector: Gaussian
  // elimination with partial pivoting of T - sig I (U has two
  // superdiagonals), three solves from a random start
  for (int q = tid; q < keep; q += nt) inv_iter<T, T>(d, e, p, sig[q], Z + q, (size_t)keep, WS + q, (size_t)keep, q);
  __syncthreads();

  // ---- 7. classical Gram-Schmidt, twice, within each cluster of close
  // eigenvalues (gaps at most 1e-3 of the unit-scaled T, the criterion of
  // LAPACK's stein): inverse-iteration vectors of eigenvalues farther apart
  // are orthogonal to about eps / gap already.  FP32 (the comparison path):
  // over all the vectors.
  int* cst = (int*)lcol;  // first vector of the cluster of q (lcol is free until step 9)
  if (tid == 0) {
    cst[0] = 0;
    for (int q = 1; q < keep; ++q)
      cst[q] = sizeof(T) == sizeof(double) && lam[q] - lam[q - 1] > (T)1e-3 ? q : (sizeof(T) == sizeof(double) ? cst[q - 1] : 0);
  }
  __syncthreads();
  for (int q = 1; q < keep; ++q) {
    const int k0 = cst[q];
    if (k0 == q) continue;  // uniform: a cluster of its own (the vector is unit-norm already)
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = k0 + wid; k < q; k += nw) {
        T s = 0;
        for (int i = lane; i < p; i += 32) s += Z[(size_t)i * keep + k] * Z[(size_t)i * keep + q];
        s = warp_sum(s);
        if (lane == 0) part[k] = s;
      }
      __syncthreads();
      for (int i = tid; i < p; i += nt) {
        T acc = Z[(size_t)i * keep + q];
        for (int k = k0; k < q; ++k) acc -= part[k] * Z[(size_t)i * keep + k];
        Z[(size_t)i * keep + q] = acc;
      }
      __syncthreads();
    }
    if (wid * 32 < p) {  // p <= nt: warp w holds rows 32w .. 32w+31
      T s = 0;
      for (int i = tid; i < p; i += nt) s += Z[(size_t)i * keep + q] * Z[(size_t)i * keep + q];
      s = warp_sum(s);
      if (lane == 0) s_red[wid] = s;
    }
    __syncthreads();
    if (wid * 32 < p) {
      T nrm2 = lane * 32 < p ? s_red[lane] : (T)0;
      nrm2 = warp_sum(nrm2);
      T sc = (T)1;
      if (lane == 0 && nrm2 > (T)0) sc = (T)1 / sqrt(nrm2);  // one lane per warp (FP64 issue is scarce)
      sc = __shfl_sync(0xffffffffu, sc, 0);
      for (int i = tid; i < p; i += nt) Z[(size_t)i * keep + q] *= sc;
    }
    __syncthreads();
  }

  // ---- 8. back-transform Y = Q Z = P_0 P_1 ... P_{p-3} Z; every thread owns
  // the rows r0, r0 + rstep, ... of column j0 at every step (rows it reads
  // in one step are the rows it wrote in the previous one: no barrier needed
  // between the update of one reflector and the dot products of the next)
  const int rstep = nt / keep, j0 = tid % keep, r0 = tid / keep;
  const bool own = r0 < rstep;
  for (int k = p - 3; k >= 0; --k) {
    const T t = tau[k];
    if (t == (T)0) continue;
    const T* vk = B + (size_t)k * ldp;
    // first owned row at or below k+1
    const int rb = r0 >= k + 1 ? r0 : r0 + ((k + 1 - r0 + rstep - 1) / rstep) * rstep;
    if (own) {
      T s = 0;
      for (int r = rb; r < p; r += rstep) s += (r == k + 1 ? (T)1 : vk[r]) * Z[(size_t)r * keep + j0];
      part[r0 * keep + j0] = s;
    }
    __syncthreads();
    if (tid < keep) {
      T s = 0;
      for (int g2 = 0; g2 < rstep; ++g2) s += part[g2 * keep + tid];
      wv[tid] = t * s;
    }
    __syncthreads();
    if (own) {
      const T sj = wv[j0];
      for (int r = rb; r < p; r += rstep) Z[(size_t)r * keep + j0] -= (r == k + 1 ? (T)1 : vk[r]) * sj;
    }
  }

  // ---- 9. Coef = L~^{-T} D^{-1/2} Y (back substitution, rows of L~ staged)
  if (own)
    for (int r = r0; r < p; r += rstep) Z[(size_t)r * keep + j0] *= rs[r];
  for (int c = tid; c < p - 1; c += nt) lcol[((p - 1) & 1) * p + c] = Lg[(p - 1) + (size_t)c * p];
  __syncthreads();
  for (int i = p - 1; i >= 1; --i) {
    const T* lr = lcol + (i & 1) * p;
    T* ln = lcol + ((i - 1) & 1) * p;
    for (int c = tid; c < i - 1; c += nt) ln[c] = Lg[(i - 1) + (size_t)c * p];
    if (own) {
      const T zi = Z[(size_t)i * keep + j0];
      for (int r = r0; r < i; r += rstep) Z[(size_t)r * keep + j0] -= lr[r] * zi;
    }
    __syncthreads();
  }
  if (own)
    for (int r = r0; r < p; r += rstep) I.Coef[r + (size_t)j0 * p] = (double)Z[(size_t)r * keep + j0];
  if (tid < keep) I.theta[tid] = (double)(lam[tid] * tn);
  if (tid == 0) {
    ctl->npos_rr = s_npos;
    ctl->rr_fail = 0;
  }
}

template __global__ void k_rr_tri<float>(Inst*, const int*, int, unsigned);
template __global__ void k_rr_tri<double>(Inst*, const int*, int, unsigned);

}  // namespace sdpg
