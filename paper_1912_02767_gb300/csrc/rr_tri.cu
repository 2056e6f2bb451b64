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
//   top `keep` eigenvalues of T by Sturm-sequence multisection, their
//   eigenvectors by inverse iteration, orthonormalized (classical Gram-
//   Schmidt, twice), back-transformed by Q
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

namespace sdpg {

namespace {

template <typename T>
struct TriK;
template <>
struct TriK<float> {
  static constexpr float piv_min = 1e-6f;           // Cholesky-QR breakdown (Gram of unit columns)
  static constexpr float eps = 5.9604645e-08f;      // unit roundoff 2^-24
  static constexpr float safmin = 1.17549435e-38f;  // smallest normal
};
template <>
struct TriK<double> {
  static constexpr double piv_min = 1e-12;
  static constexpr double eps = 1.1102230246251565e-16;  // 2^-53
  static constexpr double safmin = 2.2250738585072014e-308;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x: the
// count of negative pivots of the LDL^T factorization of T - x I (Sturm
// sequence).  A pivot smaller than pivmin in magnitude is replaced by
// -pivmin, which keeps the count monotone in x.
template <typename T>
__device__ __forceinline__ int sturm_below(const T* d, const T* e2, int p, T x, T pivmin) {
  T q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < (T)0;
  for (int i = 1; i < p; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < (T)0;
  }
  return c;
}

// Start vector of inverse iteration: uniform in [-1, 1) from the Philox
// stream keyed for this purpose (row i, vector q).
template <typename T>
__device__ __forceinline__ T start_value(int i, int q) {
  uint32_t c[4] = {(uint32_t)i, (uint32_t)q, 0x52525452u, 0u};
  philox4x32_10(c, 0x7452694Eu, 0x49544552u);
  return (T)((double)c[0] * (1.0 / 2147483648.0) - 1.0);
}

// S-section search for eigenvalues p-keep .. p-1 (ascending) of the
// tridiagonal (d, e2 = e^2): lane groups of S (a power of two <= 32) per
// eigenvalue, each lane counting at one of S interior points per step, until
// the bracket is narrower than tol.  refine = false: start from [lo0, hi0];
// refine = true: start from lam[q] -/+ lo0 (checked by two counts, else the
// whole scaled spectrum [-1.01, 1.01]).  Writes lam[q] (midpoint).
template <typename TS, typename TL>
__device__ void section_search(const TS* d, const TS* e2, int p, int keep, int S, TS tol, TS lo0, TS hi0, TS pivmin,
                               TL* lam, bool refine) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const int G = nt / S, g = tid / S, sl = tid % S;
  const unsigned gbase = (unsigned)(lane & ~(S - 1));
  const unsigned gmask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << gbase);
  for (int q = g; q < keep; q += G) {  // lanes of a group share q: group-uniform
    const int J = p - keep + q;
    TS lo = lo0, hi = hi0;
    if (refine) {
      const TS c = (TS)lam[q];
      lo = c - lo0;
      hi = c + lo0;
      const int clo = sturm_below(d, e2, p, lo, pivmin), chi = sturm_below(d, e2, p, hi, pivmin);
      if (!(clo <= J && J < chi)) {
        lo = (TS)-1.01;
        hi = (TS)1.01;
      }
    }
    for (int it = 0; it < 200 && hi - lo > tol; ++it) {
      const TS step = (hi - lo) / (TS)(S + 1);
      const int c = sturm_below(d, e2, p, lo + step * (TS)(sl + 1), pivmin);
      unsigned b = __ballot_sync(gmask, c > J) >> gbase;
      if (S < 32) b &= (1u << S) - 1u;
      const int f = __ffs(b) - 1;  // first point above eigenvalue J (-1: none)
      const TS nlo = f < 0 ? lo + step * (TS)S : (f == 0 ? lo : lo + step * (TS)f);
      const TS nhi = f < 0 ? hi : lo + step * (TS)(f + 1);
      if (nlo == lo && nhi == hi) break;  // no representable progress
      lo = nlo;
      hi = nhi;
    }
    if (sl == 0) lam[q] = (TL)((TS)0.5 * (lo + hi));
  }
}

}  // namespace

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

  // ---- 1. G = L~ D L~^T (right-looking, lower triangle of B)
  for (int t = tid; t < p * p; t += nt) {
    const int i = t % p, j = t / p;
    if (i >= j) B[i + j * ldp] = (T)I.G[t];
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const T djj = B[j + j * ldp];
    if (!(djj > (T)TriK<T>::piv_min)) {
      if (tid == 0) s_fail = j + 1;
      break;  // every thread reads the same pivot: uniform exit
    }
    // scalar work only in the warps that use it (FP64 issue is scarce)
    if (j + 1 + wid < p) {
      const T inv = (T)1 / djj;
      for (int c = j + 1 + wid; c < p; c += nw) {
        const T bc = B[c + j * ldp] * inv;
        for (int r = c + lane; r < p; r += 32) B[r + c * ldp] -= B[r + j * ldp] * bc;
      }
    }
    if (j > 0 && j + tid < p) {  // column j-1 is no longer read: scale it to L~
      const T invp = (T)1 / B[(j - 1) + (j - 1) * ldp];
      for (int r = j + tid; r < p; r += nt) B[r + (j - 1) * ldp] *= invp;
    }
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
      if (s > (T)0) {  // P = I - t v v^T with v_0 = 1 maps x to beta e_1
        const T alpha = sqrt(x0 * x0 + s);
        beta = x0 >= (T)0 ? -alpha : alpha;
        t = (beta - x0) / beta;
        scale = (T)1 / (x0 - beta);
      }
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
    {
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
    }
    __syncthreads();
    // A22 -= v w'^T + w' v^T with w' = w - K v, K = t/2 w^T v
    if (wid < r) {
      T K = lane < nw ? s_red[lane] : (T)0;
      K = warp_sum(K) * ((T)0.5 * t);
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
    const float tol32 = (dbl ? 32.0f : 4.0f) * TriK<float>::eps;
    section_search<float>(db, eb, p, keep, S2, tol32, -1.01f, 1.01f, TriK<float>::safmin, lam, false);
    if (dbl) {
      __syncthreads();
      int S4 = 4;
      while (S4 > 1 && S4 * keep > nt) S4 >>= 1;
      section_search<T>(d, e2, p, keep, S4, (T)4 * TriK<T>::eps, (T)(64.0f * TriK<float>::eps), (T)0,
                        (T)TriK<T>::safmin, lam, true);
    }
    if (tid == nt - 1) s_npos = p - sturm_below(d, e2, p, (T)0, (T)TriK<T>::safmin);
  }
  __syncthreads();
  if (tid == 0) {  // shifts at least 10 eps apart, so that equal eigenvalues get distinct vectors
    const T sep = (T)10 * TriK<T>::eps;
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
  for (int q = tid; q < keep; q += nt) {
    const T sg = sig[q], tiny = TriK<T>::eps;
    for (int i = 0; i < p; ++i) Z[(size_t)i * keep + q] = start_value<T>(i, q);
    for (int it = 0; it < 3; ++it) {
      T a = d[0] - sg, bc = p > 1 ? e[0] : (T)0, zi = Z[q];
      for (int i = 0; i + 1 < p; ++i) {
        const T ei = e[i], an = d[i + 1] - sg, en = i + 2 < p ? e[i + 1] : (T)0;
        const T zn = Z[(size_t)(i + 1) * keep + q];
        T u0, u1, u2, zr;
        if (fabs(a) >= fabs(ei)) {  // pivot on the active row
          if (a == (T)0) a = tiny;
          const T f = ei / a;
          u0 = a; u1 = bc; u2 = 0; zr = zi;
          a = an - f * bc; bc = en; zi = zn - f * zi;
        } else {  // interchange with row i+1
          const T f = a / ei;
          u0 = ei; u1 = an; u2 = en; zr = zn;
          a = bc - f * an; bc = -f * en; zi = zi - f * zn;
        }
        T* w = WS + (size_t)3 * i * keep + q;
        w[0] = u0;
        w[keep] = u1;
        w[2 * (size_t)keep] = u2;
        Z[(size_t)i * keep + q] = zr;
      }
      if (a == (T)0) a = tiny;
      T x1 = zi / a, x2 = 0, mx = fabs(x1);
      Z[(size_t)(p - 1) * keep + q] = x1;
      for (int i = p - 2; i >= 0; --i) {
        const T* w = WS + (size_t)3 * i * keep + q;
        const T xi = (Z[(size_t)i * keep + q] - w[keep] * x1 - w[2 * (size_t)keep] * x2) / w[0];
        Z[(size_t)i * keep + q] = xi;
        x2 = x1;
        x1 = xi;
        mx = fmax(mx, fabs(xi));
      }
      const T inv = mx > (T)0 && isfinite(mx) ? (T)1 / mx : (T)1;
      T s2 = 0;
      for (int i = 0; i < p; ++i) {
        const T v = Z[(size_t)i * keep + q] * inv;
        s2 += v * v;
      }
      const T sc = s2 > (T)0 ? inv / sqrt(s2) : (T)1;
      for (int i = 0; i < p; ++i) Z[(size_t)i * keep + q] *= sc;
    }
  }
  __syncthreads();

  // ---- 7. classical Gram-Schmidt, twice, over the keep vectors
  for (int q = 1; q < keep; ++q) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = wid; k < q; k += nw) {
        T s = 0;
        for (int i = lane; i < p; i += 32) s += Z[(size_t)i * keep + k] * Z[(size_t)i * keep + q];
        s = warp_sum(s);
        if (lane == 0) part[k] = s;
      }
      __syncthreads();
      for (int i = tid; i < p; i += nt) {
        T acc = Z[(size_t)i * keep + q];
        for (int k = 0; k < q; ++k) acc -= part[k] * Z[(size_t)i * keep + k];
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
      const T sc = nrm2 > (T)0 ? (T)1 / sqrt(nrm2) : (T)1;
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
