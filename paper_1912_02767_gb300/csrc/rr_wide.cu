// rr_wide.cu -- the Rayleigh-Ritz step of LOBPCG (Algorithm 3; as in
// Algorithm 2) for one wide trial subspace spread over the whole GPU, by
// tridiagonal reduction.  H = L^{-1} M L^{-T} comes from the blocked
// Cholesky factorisation and inverse with split products (rr_blocked.cu,
// oz_gemm.cu; the FP64 path: the cooperative one of rr_large.cu) and two
// products; then
//   k_trid_cluster Householder tridiagonalization of H on one thread-block
//                  cluster, H in its distributed shared memory (while it fits)
//   k_latrd_coop   otherwise, blocked: panels of reflectors on every SM, the
//                  rank-2k trailing updates as split products (mixed path)
//   k_trid_coop    or unblocked (FP64 and FP32 paths): in a working copy of
//                  precision T (L2-resident); column c belongs to CTA
//                  c mod gridDim.x; two grid barriers per step; the tail
//                  scales (d, e) to unit Gershgorin norm
//   k_trid_eig     top `keep` eigenvalues by S-section on the Sturm count
//                  (FP32 search; FP64 refinement in a second launch for
//                  T = double), the Ritz values and the positive count
//   k_trid_shift   inverse-iteration shifts (sequential prefix)
//   k_trid_invit   inverse iteration, one thread per eigenvector
//   k_trid_backtr  Y = Q Z: every CTA applies all reflectors to its own
//                  vectors (block-level reductions only); the mixed path
//                  uses the compact-WY form with split products instead
// and, by products and Cholesky launches, Cholesky-QR twice of Y and
// Coef = L^{-T} Y.
//
// Vector scratch (`vb`, T elements): d, e, e2, tau, w (p each), lam, sig
// (keep each), then doubles: tn, 1/tn, and 1024 per-CTA partial sums.
#include "kernels.h"
#include "tri_common.cuh"
#include "gridbar.cuh"
#include <cooperative_groups.h>

namespace sdpg {
using namespace tri;

template <typename T>
struct WideVec {
  T *d, *e, *e2, *tau, *w, *lam, *sig;
  double *sc, *part;
  __device__ WideVec(double* vb, int p, int keep) {
    d = (T*)vb;
    e = d + p;
    e2 = e + p;
    tau = e2 + p;
    w = tau + p;
    lam = w + p;
    sig = lam + keep;
    sc = vb + (((size_t)(5 * p + 2 * keep) * sizeof(T) + 7) / 8);
    part = sc + 2;
  }
};

__device__ __forceinline__ bool bar_failed(const GridBar* b) {
  return *(const volatile int*)&b->fail || *(const volatile int*)&b->err;
}

// block-wide sum, result returned to every thread (two barriers)
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = lane < nw ? red[lane] : (T)0;
  return warp_sum(s);
}

// Tail of the reduction (one CTA): the last 2 x 2 block into (d, e), the
// Gershgorin scaling of (d, e) to unit norm, e^2; non-finite data marks a
// breakdown.  (d, e) may come from other CTAs: read past L1.
template <typename T>
__device__ void trid_tail(const T* A, int p, WideVec<T>& V, GridBar* b) {
  __shared__ T rlo[32], rhi[32];
  __shared__ T tscal;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (tid == 0) {
    if (p >= 2) {
      V.d[p - 2] = __ldcg(A + (size_t)(p - 2) * p + (p - 2));
      V.d[p - 1] = __ldcg(A + (size_t)(p - 1) * p + (p - 1));
      V.e[p - 2] = __ldcg(A + (size_t)(p - 2) * p + (p - 1));
    } else {
      V.d[0] = __ldcg(A);
    }
  }
  __syncthreads();
  T lo = 0, hi = 0;
  int bad = 0;
  for (int i = tid; i < p; i += nt) {
    const T di = __ldcg(V.d + i);
    const T off = (i > 0 ? fabs(__ldcg(V.e + i - 1)) : (T)0) + (i + 1 < p ? fabs(__ldcg(V.e + i)) : (T)0);
    lo = fmin(lo, di - off);
    hi = fmax(hi, di + off);
    bad |= !isfinite(di) || !isfinite(off);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  bad = __syncthreads_or(bad);
  if (lane == 0) {
    rlo[wid] = lo;
    rhi[wid] = hi;
  }
  __syncthreads();
  if (tid == 0) {
    T l = 0, h = 0;
    for (int w2 = 0; w2 < nw; ++w2) {
      l = fmin(l, rlo[w2]);
      h = fmax(h, rhi[w2]);
    }
    T nrm = fmax(fabs(l), fabs(h));
    nrm = nrm > (T)0 ? nrm : (T)1;
    V.sc[0] = (double)nrm;
    V.sc[1] = 1.0 / (double)nrm;
    tscal = (T)1 / nrm;
    if (bad) atomicCAS(&b->fail, 0, -3);  // non-finite data: breakdown
  }
  __syncthreads();
  const T itn = tscal;
  for (int i = tid; i < p; i += nt) {
    V.d[i] = __ldcg(V.d + i) * itn;
    if (i + 1 < p) {
      const T ei = __ldcg(V.e + i) * itn;
      V.e[i] = ei;
      V.e2[i] = ei * ei;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_trid_tail(const T* A, int p, int keep, double* vb, GridBar* b) {
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b)) return;
  trid_tail(A, p, V, b);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_trid_coop(const double* H, T* A, int p, int keep, double* vb, GridBar* b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* vs = (T*)smraw;  // Householder vector of the step (v_0 = 1)
  T* ws = vs + p;     // w = tau A22 v of the step
  __shared__ T red[32];
  __shared__ T scal[4];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int G = gridDim.x, bid = blockIdx.x;
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b)) return;
  // working copy, symmetrized: CTA bid owns the columns c = bid mod G
  for (int c = bid; c < p; c += G)
    for (int i = tid; i < p; i += nt) A[(size_t)c * p + i] = (T)(0.5 * (H[(size_t)c * p + i] + H[(size_t)i * p + c]));
  if (!gbar(b)) return;
  for (int k = 0; k + 2 < p; ++k) {
    const int r = p - k - 1;
    const T* colk = A + (size_t)k * p + (k + 1);
    // Householder reflector P = I - t v v^T mapping x = A[k+1:, k] to beta e_1,
    // computed by every CTA from the same data
    T s = 0;
    for (int i = 1 + tid; i < r; i += nt) {
      const T x = __ldcg(colk + i);  // column k was updated by its owner: read past L1
      s += x * x;
    }
    s = block_sum(s, red);
    if (tid == 0) {
      const T x0 = __ldcg(colk);
      T beta = x0, t = 0, scale = 0;
      if (s > (T)0) {
        const T alpha = sqrt(x0 * x0 + s);
        beta = x0 >= (T)0 ? -alpha : alpha;
        t = (beta - x0) / beta;
        scale = (T)1 / (x0 - beta);
      }
      scal[0] = beta;
      scal[1] = t;
      scal[2] = scale;
    }
    __syncthreads();
    const T beta = scal[0], t = scal[1], scale = scal[2];
    for (int i = tid; i < r; i += nt) vs[i] = i == 0 ? (T)1 : __ldcg(colk + i) * scale;
    __syncthreads();
    const int cfirst = k + 1 + ((bid - (k + 1)) % G + G) % G;  // first owned column of the block
    if (t != (T)0) {
      // w_c = t A22[:, c] . v on the owned columns (symmetric: column = row)
      T pw = 0;
      for (int c = cfirst + wid * G; c < p; c += nw * G) {
        const T* col = A + (size_t)c * p + (k + 1);
        T acc = 0;
        for (int i = lane; i < r; i += 32) acc += col[i] * vs[i];
        acc = warp_sum(acc) * t;
        if (lane == 0) {
          V.w[c] = acc;
          pw += acc * vs[c - k - 1];
        }
      }
      pw = block_sum(pw, red);
      if (tid == 0) V.part[bid] = (double)pw;
    }
    if (!gbar(b)) return;  // column k read by every CTA; w and partials complete
    if (k % G == bid) {    // the owner keeps v below the subdiagonal and (d_k, e_k, tau_k)
      T* ck = A + (size_t)k * p + (k + 1);
      for (int i = 1 + tid; i < r; i += nt) ck[i] = vs[i];
      if (tid == 0) {
        V.d[k] = A[(size_t)k * p + k];
        V.e[k] = beta;
        V.tau[k] = t;
      }
    }
    if (t != (T)0) {
      if (tid < 32) {  // K = t/2 w^T v over all CTAs, fixed order
        T kk = 0;
        for (int g = lane; g < G; g += 32) kk += (T)__ldcg(V.part + g);
        kk = warp_sum(kk);
        if (lane == 0) scal[3] = kk * (T)0.5 * t;
      }
      for (int i = tid; i < r; i += nt) ws[i] = __ldcg(V.w + k + 1 + i);
      __syncthreads();
      const T K = scal[3];
      // A22[:, c] -= v w'_c + w' v_c, w' = w - K v, on the owned columns
      for (int c = cfirst + wid * G; c < p; c += nw * G) {
        T* col = A + (size_t)c * p + (k + 1);
        const int jc = c - k - 1;
        const T vc = vs[jc], wc = ws[jc] - K * vc;
        for (int i = lane; i < r; i += 32) col[i] -= vs[i] * wc + (ws[i] - K * vs[i]) * vc;
      }
    }
    if (!gbar(b)) return;
  }
  if (bid != 0) return;
  trid_tail(A, p, V, b);  // CTA 0
}

// One panel [j0, j1) of the blocked Householder tridiagonalization of the
// symmetric A (p x p, ld p, full storage), for the mixed path (its trailing
// updates run on the tensor cores).  For every column k of the panel (c =
// k - j0), with V, W the panel's earlier Householder vectors and their
// w-vectors (W kept before the correction w -= K v, K per column in Kc):
//   (a) column k below the diagonal minus the earlier rank-2 terms
//       V W[k, :]^T + W V[k, :]^T, on this CTA's rows (i = bid mod G);
//   (b) the reflector P = I - t v v^T of the updated column (every CTA,
//       same data, fixed order), s = A22 v on the owned columns (A22 not yet
//       updated by the panel: columns right of k are untouched here), and
//       the partial sums of W^T v, V^T v over the owned rows;
//   (c) w = t (s - V (W^T v) - W (V^T v)) on the owned entries, stored with
//       v into the panels (v also below the subdiagonal of A for the
//       back-transform); K = t/2 w^T v.
// Three grid barriers per column; the host then applies A22 -= V W^T +
// W V^T (W corrected by K) as two FP64-accurate products.  pt holds per CTA
// [norm^2, w^T v, W^T v (kLatrdNb), V^T v (kLatrdNb)] partial sums.
// Dynamic shared memory: (p + kLatrdOwn + 3 kLatrdNb) doubles.
__global__ void __launch_bounds__(1024) k_latrd_coop(double* A, int p, int keep, int j0, int j1, double* Vp,
                                                      double* Wp, double* Kg, double* pt, double* vb, GridBar* b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* vs = (double*)smraw;  // Householder vector of the step (v_0 = 1)
  double* sj = vs + p;          // A22 v on the owned columns
  double* y1 = sj + kLatrdOwn;  // W^T v
  double* y2 = y1 + kLatrdNb;   // V^T v
  double* Kc = y2 + kLatrdNb;   // K of the panel's columns
  __shared__ double red[32];
  __shared__ double scal[2];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int G = gridDim.x, bid = blockIdx.x;
  const int PT = 2 + 2 * kLatrdNb;
  WideVec<double> V(vb, p, keep);
  if (bar_failed(b)) return;
  if (j1 - j0 > kLatrdNb || (p - j0 + G - 1) / G > kLatrdOwn) {  // launch sized for another width: refuse
    if (bid == 0 && tid == 0) atomicCAS(&b->fail, 0, -4);
    return;
  }
  for (int k = j0; k < j1; ++k) {
    const int c = k - j0, r = p - k - 1;
    // (a) owned rows i >= k of column k
    const int ifirst = k + ((bid - k) % G + G) % G;
    double pn = 0.0;
    for (int i = ifirst + wid * G; i < p; i += nw * G) {
      double acc = 0.0;
      for (int q = lane; q < c; q += 32) {
        const double vk = __ldcg(Vp + k + (size_t)q * p), wk = __ldcg(Wp + k + (size_t)q * p) - Kc[q] * vk;
        const double vi = __ldcg(Vp + i + (size_t)q * p), wi = __ldcg(Wp + i + (size_t)q * p) - Kc[q] * vi;
        acc += vi * wk + wi * vk;
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        const double x = __ldcg(A + i + (size_t)k * p) - acc;
        A[i + (size_t)k * p] = x;
        if (i >= k + 2) pn += x * x;
      }
    }
    pn = block_sum(pn, red);
    if (tid == 0) pt[(size_t)bid * PT] = pn;
    if (!gbar(b)) return;
    // (b) the reflector, from every CTA's partial norm (one warp, fixed order)
    if (wid == 0) {
      double sn = 0.0;
      for (int g = lane; g < G; g += 32) sn += __ldcg(pt + (size_t)g * PT);
      sn = warp_sum(sn);
      if (lane == 0) red[0] = sn;
    }
    __syncthreads();
    if (tid == 0) {
      const double sn = red[0];
      const double x0 = __ldcg(A + (k + 1) + (size_t)k * p);
      double beta = x0, t = 0.0, scale = 0.0;
      if (sn > 0.0) {
        const double alpha = sqrt(x0 * x0 + sn);
        beta = x0 >= 0.0 ? -alpha : alpha;
        t = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
      }
      scal[0] = t;
      scal[1] = scale;
      if (bid == 0) {
        V.d[k] = __ldcg(A + k + (size_t)k * p);
        V.e[k] = beta;
        V.tau[k] = t;
      }
    }
    __syncthreads();
    const double t = scal[0], scale = scal[1];
    for (int i = tid; i < r; i += nt) vs[i] = i == 0 ? 1.0 : __ldcg(A + (k + 1 + i) + (size_t)k * p) * scale;
    __syncthreads();
    const int jfirst = (k + 1) + ((bid - (k + 1)) % G + G) % G;
    for (int j = jfirst + wid * G, oj = wid; j < p; j += nw * G, oj += nw) {
      const double* col = A + (size_t)j * p + (k + 1);
      double acc = 0.0;
      for (int i = lane; i < r; i += 32) acc += col[i] * vs[i];
      acc = warp_sum(acc);
      if (lane == 0) sj[oj] = acc;
    }
    for (int q = wid; q < c; q += nw) {
      double a1 = 0.0, a2 = 0.0;
      for (int i = jfirst + lane * G; i < p; i += 32 * G) {
        const double vi = vs[i - k - 1];
        const double vp = __ldcg(Vp + i + (size_t)q * p), wf = __ldcg(Wp + i + (size_t)q * p) - Kc[q] * vp;
        a1 += wf * vi;
        a2 += vp * vi;
      }
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == 0) {
        pt[(size_t)bid * PT + 2 + q] = a1;
        pt[(size_t)bid * PT + 2 + kLatrdNb + q] = a2;
      }
    }
    if (!gbar(b)) return;
    // (c) w on the owned entries
    for (int q = wid; q < c; q += nw) {  // a warp per q, lanes over the CTAs
      double a1 = 0.0, a2 = 0.0;
      for (int g = lane; g < G; g += 32) {
        a1 += __ldcg(pt + (size_t)g * PT + 2 + q);
        a2 += __ldcg(pt + (size_t)g * PT + 2 + kLatrdNb + q);
      }
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == 0) {
        y1[q] = a1;
        y2[q] = a2;
      }
    }
    __syncthreads();
    double pw = 0.0;
    for (int j = jfirst + wid * G, oj = wid; j < p; j += nw * G, oj += nw) {
      double corr = 0.0;
      for (int q = lane; q < c; q += 32) {
        const double vp = __ldcg(Vp + j + (size_t)q * p), wf = __ldcg(Wp + j + (size_t)q * p) - Kc[q] * vp;
        corr += vp * y1[q] + wf * y2[q];
      }
      corr = warp_sum(corr);
      if (lane == 0) {
        const double w = t * (sj[oj] - corr), vj = vs[j - k - 1];
        Wp[j + (size_t)c * p] = w;
        Vp[j + (size_t)c * p] = vj;
        if (j >= k + 2) A[j + (size_t)k * p] = vj;  // Householder vector below the subdiagonal
        pw += w * vj;
      }
    }
    pw = block_sum(pw, red);
    if (tid == 0) pt[(size_t)bid * PT + 1] = pw;
    if (!gbar(b)) return;
    if (wid == 0) {
      double sw = 0.0;
      for (int g = lane; g < G; g += 32) sw += __ldcg(pt + (size_t)g * PT + 1);
      sw = warp_sum(sw);
      if (lane == 0) {
        Kc[c] = 0.5 * t * sw;
        if (bid == 0) Kg[c] = Kc[c];
      }
    }
    __syncthreads();
  }
}

// W[:, c] -= K_c V[:, c] for rows r0.. of the panel's nc columns
__global__ void k_latrd_wfinal(const double* Vp, double* Wp, const double* Kg, int p, int r0, int nc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int rows = p - r0;
  if (t >= (long long)rows * nc) return;
  const int i = r0 + (int)(t % rows), c = (int)(t / rows);
  Wp[i + (size_t)c * p] -= Kg[c] * Vp[i + (size_t)c * p];
}

// A = (H + H^T) / 2 (p x p, ld p)
__global__ void k_sym_copy(const double* H, double* A, int p) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p * p) return;
  const int i = (int)(t % p), j = (int)(t / p);
  A[t] = 0.5 * (H[t] + H[(size_t)i * p + j]);
}

// Top `keep` eigenvalues of the scaled tridiagonal.  TS is the precision of
// the search: float for the wide search, T = double for the refinement
// (refine = 1, from the FP32 bracket).  The last launch of a step
// (final = 1) writes the Ritz values theta = tn lam and the positive count.
template <typename TS, typename T>
__global__ void __launch_bounds__(256) k_trid_eig(double* vb, int p, int keep, int S, int refine, int final,
                                                  double* theta, int* npos, const GridBar* b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TS* ds = (TS*)smraw;
  TS* e2s = ds + p;
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < p; i += nt) {
    ds[i] = (TS)V.d[i];
    e2s[i] = i + 1 < p ? (TS)V.e2[i] : (TS)0;
  }
  __syncthreads();
  const int gpb = nt / S;
  const TS tol = refine ? (TS)4 * K<TS>::eps : (sizeof(T) == sizeof(float) ? 4 : 32) * (TS)K<float>::eps;
  if (refine)
    section_search<TS, T>(ds, e2s, p, keep, S, blockIdx.x * gpb + tid / S, gridDim.x * gpb, tol,
                          (TS)(64.0f * K<float>::eps), (TS)0, K<TS>::safmin, V.lam, true);
  else
    section_search<TS, T>(ds, e2s, p, keep, S, blockIdx.x * gpb + tid / S, gridDim.x * gpb, tol, (TS)-1.01,
                          (TS)1.01, K<TS>::safmin, V.lam, false);
  if (!final) return;
  __syncthreads();
  // the lanes that wrote lam[q] publish theta[q] (same group mapping)
  const int g = blockIdx.x * gpb + tid / S;
  if (tid % S == 0)
    for (int q = g; q < keep; q += gridDim.x * gpb) theta[q] = (double)V.lam[q] * V.sc[0];
  if (blockIdx.x == 0 && tid == 0) {
    const T* d = V.d;
    const T* e2 = V.e2;
    *npos = p - sturm_below(d, e2, p, (T)0, (T)K<T>::safmin);
  }
}

// Inverse-iteration shifts: at least 10 eps apart, so that equal
// eigenvalues get distinct vectors.
template <typename T>
__global__ void k_trid_shift(double* vb, int p, int keep, const GridBar* b) {
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b) || threadIdx.x != 0 || blockIdx.x != 0) return;
  const T sep = (T)10 * K<T>::eps;
  T prev = V.lam[0];
  V.sig[0] = prev;
  for (int q = 1; q < keep; ++q) {
    T s = V.lam[q];
    if (s < prev + sep) s = prev + sep;
    V.sig[q] = s;
    prev = s;
  }
}

// One thread per eigenvector: Z[:, q] (column-major, ld p, FP64 storage).
template <typename T>
__global__ void __launch_bounds__(128) k_trid_invit(double* vb, int p, int keep, double* Z, T* WS, const GridBar* b) {
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= keep) return;
  inv_iter<T, double>(V.d, V.e, p, V.sig[q], Z + (size_t)q * p, 1, WS + q, (size_t)keep, q);
}

// Y = Q Z = P_0 P_1 ... P_{p-3} Z for the vectors [q0, q0 + nv) of this CTA
// (nv <= kTridBacktrNv), held in shared memory for the whole product; the
// reflectors stream through a triple buffer (v_{k-1} is fetched while v_k is
// applied, and is never written while a slower thread still reads v_{k+1}).
// Thread t owns the rows t, t + nt, ... of every vector, so no barrier
// separates the update by one reflector from the dot products of the next.
// Dynamic shared memory: rr_backtr_smem_bytes(p, nv, sizeof(T)).
template <typename T>
__global__ void __launch_bounds__(256) k_trid_backtr(const T* A, double* vb, int p, int keep, double* Y, int nv,
                                                     const GridBar* b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T red[8][kTridBacktrNv];
  __shared__ T sj[kTridBacktrNv];
  WideVec<T> V(vb, p, keep);
  if (bar_failed(b)) return;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int q0 = blockIdx.x * nv, nq = min(nv, keep - q0);
  if (nq <= 0) return;
  T* Ys = (T*)smraw;                // nq x p
  T* vbuf = Ys + (size_t)nv * p;    // 3 x p
  T* taus = vbuf + (size_t)3 * p;   // p
  double* Yb = Y + (size_t)q0 * p;
  for (int j = 0; j < nq; ++j)
    for (int i = tid; i < p; i += nt) Ys[(size_t)j * p + i] = (T)Yb[(size_t)j * p + i];
  for (int i = tid; i < p; i += nt) taus[i] = i + 2 < p ? V.tau[i] : (T)0;
  if (p >= 3) {
    const int k = p - 3;
    T* vn = vbuf + (size_t)(k % 3) * p;
    for (int i = k + 1 + tid; i < p; i += nt) vn[i] = i == k + 1 ? (T)1 : A[(size_t)k * p + i];
  }
  __syncthreads();
  for (int k = p - 3; k >= 0; --k) {
    if (k > 0) {  // fetch v_{k-1} (rows >= k) into the next buffer
      T* vn = vbuf + (size_t)((k - 1) % 3) * p;
      for (int i = k + tid; i < p; i += nt) vn[i] = i == k ? (T)1 : A[(size_t)(k - 1) * p + i];
    }
    const T t = taus[k];
    if (t == (T)0) {
      __syncthreads();  // keeps the buffer rotation in step
      continue;
    }
    const T* vs = vbuf + (size_t)(k % 3) * p;
    const int i0 = tid >= k + 1 ? tid : tid + ((k + 1 - tid + nt - 1) / nt) * nt;
    T acc[kTridBacktrNv];
#pragma unroll
    for (int j = 0; j < kTridBacktrNv; ++j) acc[j] = 0;
    for (int i = i0; i < p; i += nt) {
      const T vi = vs[i];
#pragma unroll
      for (int j = 0; j < kTridBacktrNv; ++j)
        if (j < nq) acc[j] += vi * Ys[(size_t)j * p + i];
    }
#pragma unroll
    for (int j = 0; j < kTridBacktrNv; ++j) {
      if (j >= nq) break;
      const T s = warp_sum(acc[j]);
      if (lane == 0) red[wid][j] = s;
    }
    __syncthreads();
    if (tid < nq) {
      T s = 0;
      for (int w2 = 0; w2 < nw; ++w2) s += red[w2][tid];
      sj[tid] = t * s;
    }
    __syncthreads();
    for (int i = i0; i < p; i += nt) {
      const T vi = vs[i];
#pragma unroll
      for (int j = 0; j < kTridBacktrNv; ++j)
        if (j < nq) Ys[(size_t)j * p + i] -= vi * sj[j];
    }
  }
  __syncthreads();
  for (int j = 0; j < nq; ++j)
    for (int i = tid; i < p; i += nt) Yb[(size_t)j * p + i] = (double)Ys[(size_t)j * p + i];
}

// Householder tridiagonalization of the symmetric H (p x p, ld p, FP64) on
// ONE thread-block cluster of CL CTAs, the matrix held in the cluster's
// distributed shared memory: CTA `rank` owns the columns c = rank + CL j
// (full columns, ld p | 1).  Per column k of the reduction (Algorithm 2's
// eigenproblem of H, reduced as in Golub & Van Loan 8.3.1):
//   (a) the owner of column k forms the reflector P = I - t v v^T mapping
//       H[k+1:, k] to beta e_1 and publishes v, t in its shared memory;
//   -- cluster barrier --
//   (b) every CTA copies v (distributed shared memory reads) and forms
//       w_c = t H22[:, c] . v on its owned trailing columns (symmetric:
//       column = row), split over row segments so that every FP64 lane does
//       useful work (no warp reductions), and its share of w^T v;
//   -- cluster barrier --
//   (c) every CTA gathers w and the shares, w' = w - (t/2)(w^T v) v, and
//       updates its owned columns, H22[:, c] -= v w'_c + w' v_c.
// The step's buffers alternate by parity of k, so two cluster barriers per
// column order every remote read before the next overwrite.  The owned
// columns (Householder vectors below the subdiagonal, the last 2 x 2 block)
// are written to A (p x p, ld p) at the end, (d, e, tau) to `vb` by each
// step's owner, and CTA 0 runs the tail (scaling of (d, e)).
// Dynamic shared memory: trid_cluster_smem(p, CL) bytes.
template <int CL>
__global__ void __launch_bounds__(kTridClThreads) k_trid_cluster(const double* __restrict__ H, double* A, int p,
                                                                 int keep, double* vb, GridBar* b) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ldl = p | 1, ncl = (p + CL - 1) / CL;
  double* Al = (double*)smraw;            // ncl x ldl: owned column c = rank + CL jl at jl
  double* vbuf = Al + (size_t)ncl * ldl;  // 2 x p: the step's reflector (owner), by parity of k
  double* wbuf = vbuf + 2 * p;            // 2 x p: w_c at index c for the owned c
  double* vloc = wbuf + 2 * p;            // p: local copy of v
  double* wl = vloc + p;                  // p: gathered w, then w'
  double* scb = wl + p;                   // 2 x 4: beta, t, scale, this CTA's share of w^T v
  double* part = scb + 8;                 // kTridClThreads: segment partial sums
  double* red = part + kTridClThreads;    // 32: block reductions
  __shared__ double s_K;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  WideVec<double> V(vb, p, keep);
  if (bar_failed(b)) return;  // the record is not written while this kernel runs: uniform
  for (int jl = 0; jl < ncl; ++jl) {
    const int c = rank + CL * jl;
    if (c >= p) break;
    for (int i = tid; i < p; i += nt)
      Al[(size_t)jl * ldl + i] = 0.5 * (H[(size_t)c * p + i] + H[(size_t)i * p + c]);
  }
  cl.sync();  // every CTA of the cluster resident before the first remote access
  for (int k = 0; k + 2 < p; ++k) {
    const int r = p - k - 1, par = k & 1, o = k % CL;
    double* vb_ = vbuf + par * p;
    double* wb_ = wbuf + par * p;
    double* sc_ = scb + par * 4;
    if (o == rank) {  // (a)
      double* colk = Al + (size_t)(k / CL) * ldl + (k + 1);
      double s = 0;
      for (int i = 1 + tid; i < r; i += nt) s += colk[i] * colk[i];
      s = block_sum(s, red);
      if (tid == 0) {
        const double x0 = colk[0];
        double beta = x0, t = 0, scale = 0;
        if (s > 0.0) {
          const double alpha = sqrt(x0 * x0 + s);
          beta = x0 >= 0.0 ? -alpha : alpha;
          t = (beta - x0) / beta;
          scale = 1.0 / (x0 - beta);
        }
        sc_[0] = beta;
        sc_[1] = t;
        sc_[2] = scale;
        V.d[k] = colk[-1];
        V.e[k] = beta;
        V.tau[k] = t;
      }
      __syncthreads();
      const double scale = sc_[2];
      for (int i = tid; i < r; i += nt) {
        const double v = i == 0 ? 1.0 : colk[i] * scale;
        vb_[i] = v;
        if (i > 0) colk[i] = v;  // kept below the subdiagonal for the back-transform
      }
    }
    cl.sync();  // reflector k published
    const double* rv = cl.map_shared_rank(vb_, o);
    const double t = *cl.map_shared_rank(sc_ + 1, o);  // the same value in every CTA
    for (int i = tid; i < r; i += nt) vloc[i] = rv[i];
    const int cf = k + 1 + ((rank - (k + 1)) % CL + CL) % CL;  // first owned trailing column
    const int nc = cf < p ? (p - 1 - cf) / CL + 1 : 0;
    __syncthreads();
    if (t != 0.0 && nc > 0) {  // (b), uniform in the CTA
      const int nseg = max(1, min(64, nt / nc));
      for (int q = tid; q < nc * nseg; q += nt) {
        const int a = q / nseg, g = q % nseg;
        const double* col = Al + (size_t)((cf + a * CL) / CL) * ldl + (k + 1);
        double acc = 0;
        for (int i = g; i < r; i += nseg) acc += col[i] * vloc[i];
        part[q] = acc;
      }
      __syncthreads();
      double pk = 0;
      for (int a = tid; a < nc; a += nt) {
        double w = 0;
        for (int g = 0; g < nseg; ++g) w += part[a * nseg + g];
        w *= t;
        const int c = cf + a * CL;
        wb_[c] = w;
        pk += w * vloc[c - k - 1];
      }
      pk = block_sum(pk, red);
      if (tid == 0) sc_[3] = pk;
    } else if (tid == 0) {
      sc_[3] = 0.0;
    }
    cl.sync();  // w entries and shares published
    if (t != 0.0) {  // (c), uniform in the cluster
      for (int i = tid; i < r; i += nt) {
        const int g = k + 1 + i;
        wl[i] = *cl.map_shared_rank(wb_ + g, g % CL);
      }
      if (tid == 0) {
        double kk = 0;
        for (int o2 = 0; o2 < CL; ++o2) kk += *cl.map_shared_rank(sc_ + 3, o2);  // fixed order
        s_K = 0.5 * t * kk;
      }
      __syncthreads();
      const double K = s_K;
      for (int i = tid; i < r; i += nt) wl[i] -= K * vloc[i];
      __syncthreads();
      for (int a = wid; a < nc; a += nw) {
        const int c = cf + a * CL, jc = c - k - 1;
        double* col = Al + (size_t)(c / CL) * ldl + (k + 1);
        const double vc = vloc[jc], wc = wl[jc];
        for (int i = lane; i < r; i += 32) col[i] -= vloc[i] * wc + wl[i] * vc;
      }
      __syncthreads();
    }
  }
  for (int jl = 0; jl < ncl; ++jl) {
    const int c = rank + CL * jl;
    if (c >= p) break;
    for (int i = tid; i < p; i += nt) A[(size_t)c * p + i] = Al[(size_t)jl * ldl + i];
  }
  __threadfence();
  cl.sync();  // A and (d, e, tau) complete; no remote access after this point
  if (rank != 0) return;
  trid_tail(A, p, V, b);
}

// Largest p whose owned columns fit one CTA of a CL-CTA cluster.
int trid_cluster_max_p(int cl) {
  int p = 3;
  while (trid_cluster_smem(p + 1, cl) <= kTridClSmemMax) ++p;
  return p;
}

template <int CL>
static int trid_cluster_ready() {
  static int ok = -1;
  if (ok >= 0) return ok;
  ok = 0;
  auto k = k_trid_cluster<CL>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTridClSmemMax) != cudaSuccess ||
      (CL > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return ok;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(kTridClThreads);
  cfg.dynamicSmemBytes = kTridClSmemMax;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclu = 0;
  if (cudaOccupancyMaxActiveClusters(&nclu, k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return ok;
  }
  ok = nclu > 0 ? 1 : 0;
  return ok;
}

// Cluster width for a reduction of width p: 16 CTAs where the GPU schedules
// such clusters, else 8; 0 when p exceeds what the cluster's shared memory
// holds.
int trid_cluster_width(int p) {
  static int m16 = -1, m8 = -1;
  if (m8 < 0) {
    m16 = trid_cluster_ready<16>() ? trid_cluster_max_p(16) : 0;
    m8 = trid_cluster_ready<8>() ? trid_cluster_max_p(8) : 0;
  }
  if (p <= m16) return 16;
  if (p <= m8) return 8;
  return 0;
}

int trid_cluster(cudaStream_t s, int cl, const double* H, double* A, int p, int keep, double* vb, GridBar* b) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kTridClThreads);
  cfg.dynamicSmemBytes = trid_cluster_smem(p, cl);
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cl == 16 ? cudaLaunchKernelEx(&cfg, k_trid_cluster<16>, H, A, p, keep, vb, b)
                           : cudaLaunchKernelEx(&cfg, k_trid_cluster<8>, H, A, p, keep, vb, b);
  return e == cudaSuccess ? 0 : -1;
}

template __global__ void k_trid_coop<float>(const double*, float*, int, int, double*, GridBar*);
template __global__ void k_trid_coop<double>(const double*, double*, int, int, double*, GridBar*);
template __global__ void k_trid_tail<double>(const double*, int, int, double*, GridBar*);
template __global__ void k_trid_eig<float, float>(double*, int, int, int, int, int, double*, int*, const GridBar*);
template __global__ void k_trid_eig<float, double>(double*, int, int, int, int, int, double*, int*, const GridBar*);
template __global__ void k_trid_eig<double, double>(double*, int, int, int, int, int, double*, int*, const GridBar*);
template __global__ void k_trid_shift<float>(double*, int, int, const GridBar*);
template __global__ void k_trid_shift<double>(double*, int, int, const GridBar*);
template __global__ void k_trid_invit<float>(double*, int, int, double*, float*, const GridBar*);
template __global__ void k_trid_invit<double>(double*, int, int, double*, double*, const GridBar*);
template __global__ void k_trid_backtr<float>(const float*, double*, int, int, double*, int, const GridBar*);
template __global__ void k_trid_backtr<double>(const double*, double*, int, int, double*, int, const GridBar*);

}  // namespace sdpg
