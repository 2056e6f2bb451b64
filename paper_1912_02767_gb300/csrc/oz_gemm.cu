// oz_gemm.cu -- FP64-accurate dense products C = alpha op(A) op(B) + beta C
// on the sm_103a tensor cores, for the Rayleigh-Ritz step of LOBPCG
// (Algorithm 2 inside Algorithm 3: the Grams S^T S and S^T A S of the
// Cholesky-QR orthonormalisation, the products forming H = L^{-1} M L^{-T},
// the Ritz coefficients and the block update S W).
//
// Arithmetic: the error-free splitting of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012), in its fixed-point form with per-row scaling
// (Mukunoki, Ozaki, Ogita, Imamura, "DGEMM using Tensor Cores, and Its
// Accurate and Reproducible Versions", ISC 2020), written here for bf16
// tcgen05 MMAs with FP32 accumulation in tensor memory:
//
//  * every row of op(A) (column of op(B)) gets a power-of-two scale 2^e with
//    max |x| < 2^e; x 2^-e is rounded to T/2^48 (T an integer, |error| <=
//    2^-49) and T is written as six signed base-256 digits q_1..q_6 (|q_1|
//    <= 256, |q_s| <= 128 after rounding to nearest), all exact in bf16;
//    slice s holds a_s = q_s 2^{-8(s-1)}, so x = 2^{e-8} sum_s a_s;
//  * the product keeps the pairs (s, t) with s + t <= 7 (21 MMAs per
//    k-step); pairs of equal d = s + t share the power of two 2^{-8(d-2)},
//    so each of the accumulators d = 2, 3, 4, 5 holds integers times that
//    power and stays exact in FP32 while |sum| <= 2^24, which holds for
//    128-deep chunks of K; the pairs d = 6, 7 share one accumulator whose
//    FP32 rounding is below 2^-48 of the leading term;
//  * after every 128-deep chunk the epilogue warps move the accumulators
//    into two int64 fixed-point words per output (exact integer sums, so
//    split-K partials also add exactly, in any order), and at the end
//    C = alpha 2^{e_m + f_n - 40} (hi + lo 2^-24) + beta C.
//
// Error bound: the dropped digit pairs and the 2^-49 rounding of each
// operand give |C - op(A)op(B)| <= K 2^-44 max_k|a_mk| max_k|b_kn| (plus
// the last rounding to FP64), against K^2 2^-53 max|a| max|b| for an FP64
// dot product's worst case.  Non-finite inputs make the affected outputs
// NaN.
//
// Per CTA: a 128 x 64 output tile; warp 8 issues the TMA loads (each B
// k-tile's six slices together, double-buffered; the A slices one at a
// time through a six-stage ring), warp 9 issues the MMAs, warps 0-7 drain
// tensor memory.  Every wait is bounded in time as in tc_gemm.cu, with the
// same drain of copies and MMAs in flight before tensor memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace sdpg {
using namespace tc;

constexpr int OZ_S = 6;                                  // slices per operand
constexpr int OZ_BN = 64;                                // output tile columns
constexpr int OZ_NACC = 5;                               // accumulators d = 2, 3, 4, 5 and d >= 6
constexpr int OZ_CHUNK = 2;                              // k-tiles per exact chunk (K = 128)
constexpr int OZ_ASTAGES = 6;
constexpr int OZ_BSTAGES = 2;
constexpr int OZ_A_BYTES = BM * BK * 2;                  // one slice of an A k-tile: 16 KiB
constexpr int OZ_B_BYTES = OZ_BN * BK * 2;               // one slice of a B k-tile: 8 KiB
constexpr int OZ_BSTAGE_BYTES = OZ_S * OZ_B_BYTES;       // 48 KiB
constexpr size_t OZ_SMEM = (size_t)OZ_ASTAGES * OZ_A_BYTES + (size_t)OZ_BSTAGES * OZ_BSTAGE_BYTES + 1024;
constexpr int OZ_THREADS = 320;                          // 8 epilogue warps, producer, MMA issuer
constexpr int OZ_BAD_EXP = 0x7fffffff;                   // row/column holds a non-finite value

struct OzParams {
  int M, N, K;
  int ktiles_per, splits;
  double alpha, beta;
  double* C;
  int ldc;
  const int* ea;        // M row scales of op(A)
  const int* eb;        // N column scales of op(B)
  long long* ws;        // splits > 1: 2 M N int64 (hi, lo), zeroed
  int* err;
  unsigned long long limit_ns;
};

// ---------------------------------------------------------------------------
// scales and slices.  Row r of op(X) (R rows of K elements): element k at
// X[r * rs + k * ks].
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// e[r] = E + 1 for the largest |x| = m 2^E (m in [1,2)), so max |x| < 2^e;
// 0 for a zero row; OZ_BAD_EXP when the row holds Inf or NaN
__global__ void k_oz_rowexp(const double* X, long long rs, long long ks, int R, int K, int* e) {
  __shared__ unsigned long long red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32;
  unsigned long long mx = 0;
  if (rs == 1) {  // consecutive rows are contiguous: lanes along rows
    const int r = r0 + tx;
    if (r < R)
      for (int k = ty; k < K; k += 8) mx = max(mx, abs_bits(X[(long long)r + (long long)k * ks]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
      for (int j = 1; j < 8; ++j) mx = max(mx, red[j][tx]);
      if (r < R) {
        const int be = (int)((mx >> 52) & 0x7ff);
        e[r] = be == 0x7ff ? OZ_BAD_EXP : (mx == 0 ? 0 : (be == 0 ? -1021 : be - 1022));
      }
    }
  } else {  // contiguous along k: a warp per row
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr;
      if (r >= R) break;
      unsigned long long m = 0;
      for (int k = tx; k < K; k += 32) m = max(m, abs_bits(X[(long long)r * rs + (long long)k * ks]));
      for (int o = 16; o; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
      if (tx == 0) {
        const int be = (int)((m >> 52) & 0x7ff);
        e[r] = be == 0x7ff ? OZ_BAD_EXP : (m == 0 ? 0 : (be == 0 ? -1021 : be - 1022));
      }
    }
  }
}

// out[s][r][k] (plane stride R*kld, row stride kld) = a_s of X(r, k); a
// 32 x 64 tile per CTA, staged in shared memory so that both the read (along
// r or k) and the write (along k) are coalesced
__global__ void __launch_bounds__(256) k_oz_slice(const double* X, long long rs, long long ks, int R, int K,
                                                  const int* e, __nv_bfloat16* out, int kld) {
  __shared__ double tile[32][65];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  const int tid = threadIdx.x;
  if (rs == 1) {
    for (int t = tid; t < 32 * 64; t += 256) {
      const int rr = t & 31, kk = t >> 5;
      const int r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? X[(long long)r + (long long)k * ks] : 0.0;
    }
  } else {
    for (int t = tid; t < 32 * 64; t += 256) {
      const int kk = t & 63, rr = t >> 6;
      const int r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? X[(long long)r * rs + (long long)k * ks] : 0.0;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)R * kld;
  for (int t = tid; t < 32 * 64; t += 256) {
    const int kk = t & 63, rr = t >> 6;
    const int r = r0 + rr, k = k0 + kk;
    if (r >= R || k >= K) continue;
    const int er = e[r];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(tile[rr][kk]);
    const int be = (int)((bits >> 52) & 0x7ff);
    long long T = 0;
    if (er != OZ_BAD_EXP && (bits & 0x7fffffffffffffffull) != 0) {
      // |x| = mant 2^(E-52); T = round(|x| 2^(48-e)) = round(mant 2^-(e-E+4))
      const long long mant = (long long)(bits & 0xfffffffffffffull) | (be ? (1ll << 52) : 0ll);
      const int E = be ? be - 1023 : -1022;
      const int sh = er - E + 4;  // >= 5 since |x| < 2^e
      T = sh >= 60 ? 0 : ((mant + (1ll << (sh - 1))) >> sh);
      if (bits >> 63) T = -T;
    }
    __nv_bfloat16* o = out + (size_t)r * kld + k;
#pragma unroll
    for (int s = 1; s <= OZ_S; ++s) {
      const int shift = 48 - 8 * s;
      long long q = T;
      if (shift > 0) q = (T + (1ll << (shift - 1))) >> shift;  // round to nearest (ties up)
      T -= q << shift;
      // a_s = q_s 2^(-8(s-1)): |q| <= 256, exact in bf16
      const float sc = s == 1 ? 1.0f : s == 2 ? 0x1p-8f : s == 3 ? 0x1p-16f : s == 4 ? 0x1p-24f
                       : s == 5 ? 0x1p-32f : 0x1p-40f;
      o[(size_t)(s - 1) * plane] = __float2bfloat16_rn((float)q * sc);
    }
  }
}

// ---------------------------------------------------------------------------
// the tensor-core product
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap mA,
                                                           const __grid_constant__ CUtensorMap mB, OzParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)OZ_ASTAGES * OZ_A_BYTES;
  __shared__ uint64_t a_full[OZ_ASTAGES], a_empty[OZ_ASTAGES], b_full[OZ_BSTAGES], b_empty[OZ_BSTAGES];
  __shared__ uint64_t acc_full, acc_empty, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * OZ_BN, split = blockIdx.z;
  const int ktiles_total = (P.K + BK - 1) / BK;
  const int kt0 = split * P.ktiles_per;
  const int nkt = max(0, min(P.ktiles_per, ktiles_total - kt0));
  const int nchunks = (nkt + OZ_CHUNK - 1) / OZ_CHUNK;
  const uint32_t ncols = 512;  // 5 accumulators x 64 columns, rounded to a power of two

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < OZ_ASTAGES; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < OZ_BSTAGES; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 8);  // one arrival per epilogue warp
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const unsigned long long lim = P.limit_ns ? P.limit_ns : kWaitLimitNs;
  bool drained = true;

  if (nkt > 0) {
    if (warp == 8) {
      if (lane == 0) {  // TMA producer
        int ia = 0, ib = 0;
        bool stop = false;
        for (int kt = 0; kt < nkt && !stop; ++kt) {
          const int kx = (kt0 + kt) * BK;  // a multiple of 64 elements (128 bytes)
          const int bs = kt % OZ_BSTAGES;
          if (kt >= OZ_BSTAGES && !mbar_wait(&b_empty[bs], ((kt / OZ_BSTAGES) - 1) & 1, &abort_flag, lim)) break;
          uint8_t* bst = sB + (size_t)bs * OZ_BSTAGE_BYTES;
          mbar_expect_tx(&b_full[bs], (uint32_t)OZ_BSTAGE_BYTES);
          for (int t = 0; t < OZ_S; ++t) tma_load_3d(bst + (size_t)t * OZ_B_BYTES, &mB, &b_full[bs], kx, n0, t);
          ib = kt + 1;
          for (int s = 0; s < OZ_S; ++s) {
            const int as = ia % OZ_ASTAGES;
            if (ia >= OZ_ASTAGES && !mbar_wait(&a_empty[as], ((ia / OZ_ASTAGES) - 1) & 1, &abort_flag, lim)) {
              stop = true;
              break;
            }
            mbar_expect_tx(&a_full[as], (uint32_t)OZ_A_BYTES);
            tma_load_3d(sA + (size_t)as * OZ_A_BYTES, &mA, &a_full[as], kx, m0, s);
            ++ia;
          }
        }
        // the last load issued into each stage completes its latest phase
        // whether or not the MMA side consumed it: wait for all of them
        for (int i = (ia > OZ_ASTAGES ? ia - OZ_ASTAGES : 0); i < ia; ++i)
          drained &= mbar_drain(&a_full[i % OZ_ASTAGES], (i / OZ_ASTAGES) & 1);
        for (int i = (ib > OZ_BSTAGES ? ib - OZ_BSTAGES : 0); i < ib; ++i)
          drained &= mbar_drain(&b_full[i % OZ_BSTAGES], (i / OZ_BSTAGES) & 1);
      }
    } else if (warp == 9) {
      if (lane == 0) {  // MMA issuer
        const uint32_t idesc = umma_idesc_bf16(OZ_BN);
        int ia = 0;
        bool stop = false;
        for (int kt = 0; kt < nkt && !stop; ++kt) {
          const int chunk = kt / OZ_CHUNK;
          const bool first = (kt % OZ_CHUNK) == 0;
          // the epilogue must have read the previous chunk's accumulators
          if (first && chunk > 0 && !mbar_wait(&acc_empty, (chunk - 1) & 1, &abort_flag, lim)) break;
          const int bs = kt % OZ_BSTAGES;
          if (!mbar_wait(&b_full[bs], (kt / OZ_BSTAGES) & 1, &abort_flag, lim)) break;
          tc_fence_after();
          const uint8_t* bst = sB + (size_t)bs * OZ_BSTAGE_BYTES;
          for (int s = 0; s < OZ_S; ++s) {
            const int as = ia % OZ_ASTAGES;
            if (!mbar_wait(&a_full[as], (ia / OZ_ASTAGES) & 1, &abort_flag, lim)) {
              stop = true;
              break;
            }
            tc_fence_after();
            const uint64_t adesc = umma_desc_sw128(sA + (size_t)as * OZ_A_BYTES);
            for (int t = 0; t + s < OZ_S; ++t) {  // slice pairs with (s+1) + (t+1) <= 7
              const int acc = s + t < 4 ? s + t : 4;
              const uint64_t bdesc = umma_desc_sw128(bst + (size_t)t * OZ_B_BYTES);
              const bool reset = first && s == 0 && t <= 4;  // first product into this accumulator
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
                umma_bf16(tmem + (uint32_t)(acc * OZ_BN), adesc + adv, bdesc + adv, idesc,
                          (reset && kk == 0) ? 0u : 1u);
              }
            }
            umma_commit(&a_empty[as]);  // A stage free once these MMAs have read it
            ++ia;
          }
          if (stop) break;
          umma_commit(&b_empty[bs]);
          if ((kt % OZ_CHUNK) == OZ_CHUNK - 1 || kt == nkt - 1) umma_commit(&acc_full);
        }
        umma_commit(&done_bar);  // every MMA issued (none after an abort)
      }
    } else {
      // epilogue warps: rows 32 (warp % 4) .. +31, columns 32 (warp / 4) .. +31
      const int rq = warp & 3, ch = warp >> 2;
      long long hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        if (!mbar_wait(&acc_full, c & 1, &abort_flag, lim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(rq * 32) << 16) + (uint32_t)(ch * 32);
        uint32_t r[32];
        // d = 2: integers; d = 3, 4, 5: integers times 2^-8, 2^-16, 2^-24;
        // hi in units of 2^-24
        tmem_ld32(base + 0 * OZ_BN, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << 24;
        tmem_ld32(base + 1 * OZ_BN, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 256.0f) << 16;
        tmem_ld32(base + 2 * OZ_BN, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 65536.0f) << 8;
        tmem_ld32(base + 3 * OZ_BN, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 16777216.0f);
        // d >= 6: FP32 sum, in units of 2^-48
        tmem_ld32(base + 4 * OZ_BN, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) lo[j] += __float2ll_rn(__uint_as_float(r[j]) * 281474976710656.0f);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty);
      }
      // after an abort the MMAs already issued may still run: done_bar
      // tracks them all (the issuer commits it on every exit path)
      if (!ok || abort_flag) drained &= mbar_drain(&done_bar, 0);
      if (ok && !abort_flag) {
        const int row = m0 + rq * 32 + lane;
        if (row < P.M) {
          const int er = P.ea[row];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + ch * 32 + j;
            if (col >= P.N) continue;
            if (P.splits > 1) {
              unsigned long long* w = (unsigned long long*)P.ws + 2 * ((size_t)row + (size_t)col * P.M);
              atomicAdd(w, (unsigned long long)hi[j]);
              atomicAdd(w + 1, (unsigned long long)lo[j]);
            } else {
              const int ec = P.eb[col];
              double v;
              if (er == OZ_BAD_EXP || ec == OZ_BAD_EXP) v = __longlong_as_double(0x7ff8000000000000ll);
              else v = ldexp((double)hi[j] + ldexp((double)lo[j], -24), er + ec - 40);
              double* cp = P.C + (size_t)row + (size_t)col * P.ldc;
              *cp = P.beta == 0.0 ? P.alpha * v : P.alpha * v + P.beta * *cp;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  // every thread is past its drain: nothing of this CTA is in flight (or a
  // drain itself gave up, reported as error 2)
  const int undrained = __syncthreads_or(drained ? 0 : 1);
  if (threadIdx.x == 0 && (abort_flag || undrained)) atomicMax(P.err, undrained ? 2 : 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// split-K: C = alpha 2^(e_m + f_n - 40) (hi + lo 2^-24) + beta C from the
// summed int64 words
__global__ void k_oz_finalize(const long long* ws, const int* ea, const int* eb, int M, int N, double alpha,
                              double beta, double* C, int ldc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N) return;
  const int row = (int)(t % M), col = (int)(t / M);
  const int er = ea[row], ec = eb[col];
  double v;
  if (er == OZ_BAD_EXP || ec == OZ_BAD_EXP) v = __longlong_as_double(0x7ff8000000000000ll);
  else v = ldexp((double)ws[2 * t] + ldexp((double)ws[2 * t + 1], -24), er + ec - 40);
  double* cp = C + (size_t)row + (size_t)col * ldc;
  *cp = beta == 0.0 ? alpha * v : alpha * v + beta * *cp;
}

// X = (X + X^T) / 2 for a p x p matrix (leading dimension ld)
__global__ void k_symmetrize(double* X, int p, int ld) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p * p) return;
  const int i = (int)(t % p), j = (int)(t / p);
  if (i <= j) return;
  double* a = X + (size_t)i + (size_t)j * ld;
  double* b = X + (size_t)j + (size_t)i * ld;
  const double v = 0.5 * (*a + *b);
  *a = v;
  *b = v;
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
void symmetrize(cudaStream_t s, double* X, int p, int ld) {
  if (p > 1) k_symmetrize<<<(unsigned)(((size_t)p * p + 255) / 256), 256, 0, s>>>(X, p, ld);
}

size_t oz_work_bytes(int M, int N, int K) {
  const size_t kld = (size_t)((K + 7) / 8 * 8);
  const size_t a = (size_t)OZ_S * M * kld * 2, b = (size_t)OZ_S * N * kld * 2;
  return ((a + 255) / 256 + (b + 255) / 256) * 256 + ((size_t)(M + N) * 4 + 255) / 256 * 256 +
         (size_t)M * N * 16 + 256;
}

// op(X) rows: 'N' for A (rows strided by 1, k by ld) ...
static void row_view(char op, bool is_a, int ld, long long* rs, long long* ks) {
  // op(A) row m = A(m, :) for 'N' (rs = 1, ks = ld), A(:, m) for 'T';
  // op(B) column n = B(:, n) for 'N' (rs = ld, ks = 1), B(n, :) for 'T'
  const bool strided_rows = is_a ? (op == 'N') : (op == 'T');
  if (strided_rows) {
    *rs = 1;
    *ks = ld;
  } else {
    *rs = ld;
    *ks = 1;
  }
}

int oz_gemm(cudaStream_t s, char ta, const double* A, int lda, char tb, const double* B, int ldb, int M, int N,
            int K, double alpha, double beta, double* C, int ldc, void* work, size_t work_bytes, int* err,
            int num_sms, unsigned long long limit_ns) {
  if (M < 1 || N < 1) return 0;
  if (K < 1) {  // empty product
    if (beta == 0.0)
      for (int j = 0; j < N; ++j) cudaMemsetAsync(C + (size_t)j * ldc, 0, sizeof(double) * M, s);
    else if (beta != 1.0)
      k_copy_cols<<<(unsigned)(((size_t)M * N + 255) / 256), 256, 0, s>>>(C, ldc, C, ldc, M, N, beta);
    return 0;
  }
  if (!work || work_bytes < oz_work_bytes(M, N, K)) return -2;
  const int kld = (K + 7) / 8 * 8;
  uint8_t* w = (uint8_t*)work;
  const size_t a_bytes = ((size_t)OZ_S * M * kld * 2 + 255) / 256 * 256;
  const size_t b_bytes = ((size_t)OZ_S * N * kld * 2 + 255) / 256 * 256;
  __nv_bfloat16* sa = (__nv_bfloat16*)w;
  __nv_bfloat16* sb = (__nv_bfloat16*)(w + a_bytes);
  int* ea = (int*)(w + a_bytes + b_bytes);
  int* eb = ea + M;
  long long* ws = (long long*)(w + a_bytes + b_bytes + ((size_t)(M + N) * 4 + 255) / 256 * 256);
  long long rsa, ksa, rsb, ksb;
  row_view(ta, true, lda, &rsa, &ksa);
  row_view(tb, false, ldb, &rsb, &ksb);
  k_oz_rowexp<<<(M + 31) / 32, 256, 0, s>>>(A, rsa, ksa, M, K, ea);
  k_oz_rowexp<<<(N + 31) / 32, 256, 0, s>>>(B, rsb, ksb, N, K, eb);
  k_oz_slice<<<dim3((K + 63) / 64, (M + 31) / 32), 256, 0, s>>>(A, rsa, ksa, M, K, ea, sa, kld);
  k_oz_slice<<<dim3((K + 63) / 64, (N + 31) / 32), 256, 0, s>>>(B, rsb, ksb, N, K, eb, sb, kld);
  CUtensorMap ma, mb;
  if (!make_map_bf16(&ma, sa, K, M, kld, OZ_S, BM) || !make_map_bf16(&mb, sb, K, N, kld, OZ_S, OZ_BN)) return -1;
  const int tm = (M + BM - 1) / BM, tn = (N + OZ_BN - 1) / OZ_BN;
  const int kt = (K + BK - 1) / BK;
  int splits = 1;
  while (tm * tn * splits * 2 <= num_sms && kt / (splits * 2) >= 2 * OZ_CHUNK) splits *= 2;
  int per = (kt + splits - 1) / splits;
  per = (per + OZ_CHUNK - 1) / OZ_CHUNK * OZ_CHUNK;  // whole chunks per split
  splits = (kt + per - 1) / per;
  OzParams P;
  P.M = M;
  P.N = N;
  P.K = K;
  P.ktiles_per = per;
  P.splits = splits;
  P.alpha = alpha;
  P.beta = beta;
  P.C = C;
  P.ldc = ldc;
  P.ea = ea;
  P.eb = eb;
  P.ws = ws;
  P.err = err;
  P.limit_ns = limit_ns;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM) != cudaSuccess)
      return -1;
    attr = true;
  }
  if (splits > 1) cudaMemsetAsync(ws, 0, (size_t)M * N * 16, s);
  k_oz_gemm<<<dim3(tm, tn, splits), OZ_THREADS, OZ_SMEM, s>>>(ma, mb, P);
  if (splits > 1)
    k_oz_finalize<<<(unsigned)(((size_t)M * N + 255) / 256), 256, 0, s>>>(ws, ea, eb, M, N, alpha, beta, C, ldc);
  return 0;
}

}  // namespace sdpg
