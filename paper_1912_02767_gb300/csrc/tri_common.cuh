// tri_common.cuh -- device helpers shared by the Rayleigh-Ritz eigensolvers
// that work on a symmetric tridiagonal matrix (rr_tri.cu: one CTA per
// instance; rr_wide.cu: a wide subspace across the GPU): Sturm counts,
// S-section search for selected eigenvalues (bisection on the Sturm count),
// and inverse iteration by Gaussian elimination with partial pivoting.
#pragma once
#include <math.h>
#include <string.h>
#include "common.cuh"

namespace sdpg {
namespace tri {

// Bit patterns of floating-point values (device: register moves; the host
// forms serve the CPU tests of these helpers).
__host__ __device__ __forceinline__ long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ double dfrom(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ int fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_int(x);
#else
  int b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ float ffrom(int b) {
#ifdef __CUDA_ARCH__
  return __int_as_float(b);
#else
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

template <typename T>
struct K;
template <>
struct K<float> {
  static constexpr float piv_min = 1e-6f;           // Cholesky-QR breakdown (Gram of unit columns)
  static constexpr float eps = 5.9604645e-08f;      // unit roundoff 2^-24
  static constexpr float safmin = 1.17549435e-38f;  // smallest normal
};
template <>
struct K<double> {
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
__host__ __device__ __forceinline__ int sturm_below(const T* d, const T* e2, int p, T x, T pivmin) {
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

// Number of eigenvalues of the tridiagonal (d, e2 = e^2) below x by the signs
// of its leading principal minors f_i = det(T_i - x I): f_0 = 1, f_1 = d_0 - x,
// f_{i+1} = (d_i - x) f_i - e_{i-1}^2 f_{i-1}; the count is the number of sign
// changes along f_0 .. f_p (the Sturm property of the minors; Wilkinson, The
// Algebraic Eigenvalue Problem, 5.37).  A minor that is exactly zero is
// replaced by -2^-300 times its predecessor -- its pivot f_i / f_{i-1} taken
// as tiny and negative, as the LDL^T count takes a zero pivot as -pivmin --
// so it counts as a sign change and the recurrence goes on through it (two
// zero minors in a row, as at an eigenvalue of a block split off by a zero
// e_i, would otherwise zero every later one).  A subtraction, a multiplication and an FMA per
// row and no division: on GB300 an FP64 division costs an SM sub-partition
// about twelve FP64 issue slots, and a Sturm count is one dependent chain.
// The pair (f_{i-1}, f_i) is rescaled by a power of two (integer exponent
// arithmetic) whenever the larger leaves [2^-600, 2^600]; for a matrix scaled
// to unit norm and |x| <= 1.01 a row grows the pair at most threefold.
__host__ __device__ __forceinline__ int sturm_below_minors(const double* __restrict__ d,
                                                           const double* __restrict__ e2, int p, double x) {
  double fa = 1.0, fb = d[0] - x;
  int sa = 0, c = 0;  // sign of f_{i}: 0 positive, 1 negative (f_0 = 1)
  for (int i = 0;; ++i) {
    long long bb = dbits(fb);
    if (((unsigned long long)bb << 1) == 0) {  // a zero minor
      fb = -fa * 0x1p-300;
      bb = dbits(fb);
    }
    const int sb = (int)((unsigned long long)bb >> 63);
    c += sb != sa;
    sa = sb;
    if (i + 1 >= p) break;
    const int exb = (int)((bb >> 52) & 0x7ff), exa = (int)((dbits(fa) >> 52) & 0x7ff);
    const int ex = exa > exb ? exa : exb;
    if (ex > 1023 + 600 || ex < 1023 - 600) {
      if (ex < 2047 && ex > 0) {  // not inf / nan / both zero
        const double sc = dfrom((long long)(2046 - ex) << 52);  // 2^(1023 - ex)
        fa *= sc;
        fb *= sc;
      }
    }
    const double t = e2[i] * fa;
    const double fn = fma(d[i + 1] - x, fb, -t);
    fa = fb;
    fb = fn;
  }
  return c;
}

template <typename T>
__host__ __device__ __forceinline__ int count_below(const T* d, const T* e2, int p, T x, T pivmin) {
  return sturm_below(d, e2, p, x, pivmin);
}
template <>
__host__ __device__ __forceinline__ int count_below<double>(const double* d, const double* e2, int p, double x,
                                                            double) {
  return sturm_below_minors(d, e2, p, x);
}

// Start vector of inverse iteration: uniform in [-1, 1) from the Philox
// stream keyed for this purpose (row i, vector q).
template <typename T>
__host__ __device__ __forceinline__ T start_value(int i, int q) {
  uint32_t c[4] = {(uint32_t)i, (uint32_t)q, 0x52525452u, 0u};
  philox4x32_10(c, 0x7452694Eu, 0x49544552u);
  return (T)((double)c[0] * (1.0 / 2147483648.0) - 1.0);
}

// S-section search for eigenvalues p-keep .. p-1 (ascending) of the
// tridiagonal (d, e2 = e^2) whose spectrum lies in [-1.01, 1.01]: lane
// groups of S (a power of two <= 32) per eigenvalue, each lane counting at
// one of S interior points per step, until the bracket is narrower than tol.
// Group g of `ngroups` (numbered across the whole launch by the caller)
// handles q = g, g + ngroups, ...  refine = false: start from [lo0, hi0];
// refine = true: start from lam[q] -/+ lo0 (checked by two counts, else the
// whole [-1.01, 1.01]).  Writes lam[q] (midpoint) from the group's lane 0.
template <typename TS, typename TL>
__device__ void section_search(const TS* d, const TS* e2, int p, int keep, int S, int g, int ngroups, TS tol, TS lo0,
                               TS hi0, TS pivmin, TL* lam, bool refine) {
  const int lane = threadIdx.x & 31, sl = threadIdx.x % S;
  const unsigned gbase = (unsigned)(lane & ~(S - 1));
  const unsigned gmask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << gbase);
  for (int q = g; q < keep; q += ngroups) {  // lanes of a group share q: group-uniform
    const int J = p - keep + q;
    TS lo = lo0, hi = hi0;
    if (refine) {
      const TS c = (TS)lam[q];
      lo = c - lo0;
      hi = c + lo0;
      const int clo = count_below(d, e2, p, lo, pivmin), chi = count_below(d, e2, p, hi, pivmin);
      if (!(clo <= J && J < chi)) {
        lo = (TS)-1.01;
        hi = (TS)1.01;
      }
    }
    for (int it = 0; it < 200 && hi - lo > tol; ++it) {
      const TS step = (hi - lo) / (TS)(S + 1);
      const int c = count_below(d, e2, p, lo + step * (TS)(sl + 1), pivmin);
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

// Row-interchange flag of the factorization, kept in the lowest mantissa
// bit of the stored multiplier (a change of at most one unit in its last
// place).
__host__ __device__ __forceinline__ double pack_flag(double f, int sw) {
  return dfrom((dbits(f) & ~1LL) | (long long)sw);
}
__host__ __device__ __forceinline__ float pack_flag(float f, int sw) { return ffrom((fbits(f) & ~1) | sw); }
__host__ __device__ __forceinline__ int flag_of(double f) { return (int)(dbits(f) & 1LL); }
__host__ __device__ __forceinline__ int flag_of(float f) { return fbits(f) & 1; }

// Inverse iteration for the eigenvector of the tridiagonal (d, e) nearest
// the shift sg: T - sg I = P L U is factored once by Gaussian elimination
// with partial pivoting (U has two superdiagonals; a zero pivot becomes
// tiny), then three solves (T - sg I) x = z from the Philox start vector of
// column q, normalized each time.  One reciprocal per row in the
// factorization; the solves are multiplications only.  The vector lives at
// z[i * zs] (element type TZ); per row i the factors are kept at
// w[(3 i + c) * ws]: c = 0 the multiplier (row-interchange flag in its last
// bit), 1 the reciprocal of the pivot u0, 2 the first superdiagonal u1 (the
// second, u2, is e_{i+1} after an interchange and zero otherwise).
template <typename T, typename TZ>
__host__ __device__ void inv_iter(const T* __restrict__ d, const T* __restrict__ e, int p, T sg, TZ* __restrict__ z, size_t zs,
                         T* __restrict__ w, size_t ws, int q) {
  const T tiny = K<T>::eps;
  T a = d[0] - sg, bc = p > 1 ? e[0] : (T)0;
  for (int i = 0; i + 1 < p; ++i) {
    const T ei = e[i], an = d[i + 1] - sg, en = i + 2 < p ? e[i + 1] : (T)0;
    T f, r, u1;
    int sw;
    if (fabs(a) >= fabs(ei)) {  // pivot on the active row
      if (a == (T)0) a = tiny;
      r = (T)1 / a;
      f = ei * r;
      u1 = bc;
      a = an - f * bc;
      bc = en;
      sw = 0;
    } else {  // interchange with row i+1
      r = (T)1 / ei;
      f = a * r;
      u1 = an;
      a = bc - f * an;
      bc = -f * en;
      sw = 1;
    }
    T* wi = w + (size_t)3 * i * ws;
    wi[0] = pack_flag(f, sw);
    wi[ws] = r;
    wi[2 * ws] = u1;
  }
  if (a == (T)0) a = tiny;
  const T rlast = (T)1 / a;
  for (int i = 0; i < p; ++i) z[(size_t)i * zs] = (TZ)start_value<T>(i, q);
  for (int it = 0; it < 3; ++it) {
    T zi = (T)z[0];
    for (int i = 0; i + 1 < p; ++i) {  // z <- L^{-1} P z
      const T fp = w[(size_t)3 * i * ws];
      const T zn = (T)z[(size_t)(i + 1) * zs];
      if (flag_of(fp)) {
        z[(size_t)i * zs] = (TZ)zn;
        zi = zi - fp * zn;
      } else {
        z[(size_t)i * zs] = (TZ)zi;
        zi = zn - fp * zi;
      }
    }
    T x1 = zi * rlast, x2 = 0, mx = fabs(x1);
    z[(size_t)(p - 1) * zs] = (TZ)x1;
    for (int i = p - 2; i >= 0; --i) {  // U x = z
      const T* wi = w + (size_t)3 * i * ws;
      const T u2 = flag_of(wi[0]) && i + 2 < p ? e[i + 1] : (T)0;
      const T xi = ((T)z[(size_t)i * zs] - wi[2 * ws] * x1 - u2 * x2) * wi[ws];
      z[(size_t)i * zs] = (TZ)xi;
      x2 = x1;
      x1 = xi;
      mx = fmax(mx, fabs(xi));
    }
    const T inv = mx > (T)0 && isfinite(mx) ? (T)1 / mx : (T)1;
    T s2 = 0;
    for (int i = 0; i < p; ++i) {
      const T v = (T)z[(size_t)i * zs] * inv;
      s2 += v * v;
    }
    const T sc = s2 > (T)0 ? inv / sqrt(s2) : (T)1;
    for (int i = 0; i < p; ++i) z[(size_t)i * zs] = (TZ)((T)z[(size_t)i * zs] * sc);
  }
}

}  // namespace tri
}  // namespace sdpg
