// tc_gemm.cu -- the LOBPCG block product A X (Algorithm 3: A X^k, A R^k)
// on the sm_103a tensor cores, in split-BF16 x3 arithmetic:
//
//   W = W_hi + W_lo,  B = B_hi + B_lo  (each part bf16, round to nearest)
//   W B ~= W_hi B_hi + W_hi B_lo + W_lo B_hi      (FP32 accumulation)
//
// which keeps about 16 significant bits of each operand (the dropped
// W_lo B_lo term is 2^-18 relative).  Per CTA: a 128 x BN output tile in
// TMEM, K streamed in 64-wide (128-byte) slices by TMA with 128-byte
// swizzle through a multi-stage mbarrier pipeline; one thread issues
// tcgen05.mma (kind::f16, bf16 inputs, M = 128, N = BN); the epilogue
// reads TMEM with tcgen05.ld.  Split-K over blockIdx.z spreads a single
// large product over all SMs; partials are reduced in a second kernel.
//
// Every mbarrier wait is bounded in time (TcParams::limit_ns, else
// kWaitLimitNs); on expiry the kernel records the error in *err and skips
// the rest of its work, but before the CTA releases its tensor memory it
// still waits (bounded by kDrainLimitNs) for the MMAs it issued and the
// producer waits for the TMA loads it issued, so no asynchronous copy or
// MMA outlives the CTA's shared or tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace sdpg {

using namespace tc;
static constexpr int TC_BM = tc::BM;
static constexpr int TC_BK = tc::BK;                   // bf16 elements per 128-byte row
static constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;   // 16 KiB

struct TcParams {
  int M, N, K;        // output rows (n), output columns (block width), reduction length (n)
  int splits;         // K splits over blockIdx.z
  int ktiles_per;     // k-tiles per split
  int bn;             // N tile (multiple of 16, <= 256)
  int stages;
  double alpha;
  double* out;        // FP64 column-major M x N (ld ldo) when splits == 1
  int ldo;
  float* part;        // FP32 partials: part[(s*N + col)*M + row] when splits > 1
  int* err;
  unsigned long long limit_ns;  // wait limit (0: kWaitLimitNs)
};

__global__ void __launch_bounds__(128, 1) k_tc_wprod(const __grid_constant__ CUtensorMap mWhi,
                                                     const __grid_constant__ CUtensorMap mWlo,
                                                     const __grid_constant__ CUtensorMap mBhi,
                                                     const __grid_constant__ CUtensorMap mBlo, TcParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[4], empty_bar[4], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * P.bn, split = blockIdx.z;
  const int bn = P.bn, stages = P.stages;
  const int b_bytes = bn * TC_BK * 2;
  const int stage_bytes = 2 * TC_A_BYTES + 2 * b_bytes;
  const int kt0 = split * P.ktiles_per;
  const int ktiles_total = (P.K + TC_BK - 1) / TC_BK;
  const int nkt = min(P.ktiles_per, ktiles_total - kt0);
  uint32_t ncols = 32;
  while ((int)ncols < bn) ncols <<= 1;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  const unsigned long long lim = P.limit_ns ? P.limit_ns : kWaitLimitNs;
  bool drained = true;
  if (nkt > 0) {
    if (warp == 0 && lane == 0) {
      // TMA producer
      int issued = 0;
      for (int it = 0; it < nkt; ++it) {
        const int s = it % stages;
        if (it >= stages && !mbar_wait(&empty_bar[s], ((it / stages) - 1) & 1, &abort_flag, lim)) break;
        uint8_t* st = smem + (size_t)s * stage_bytes;
        mbar_expect_tx(&full_bar[s], (uint32_t)stage_bytes);
        const int kx = (kt0 + it) * TC_BK;  // multiple of 64 elements = 128 bytes
        tma_load_2d(st, &mWhi, &full_bar[s], kx, m0);
        tma_load_2d(st + TC_A_BYTES, &mWlo, &full_bar[s], kx, m0);
        tma_load_2d(st + 2 * TC_A_BYTES, &mBhi, &full_bar[s], kx, n0);
        tma_load_2d(st + 2 * TC_A_BYTES + b_bytes, &mBlo, &full_bar[s], kx, n0);
        issued = it + 1;
      }
      // the last load issued into each stage completes its latest phase
      // whether or not the MMA side consumed it: wait for all of them
      for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
        drained &= mbar_drain(&full_bar[it % stages], (it / stages) & 1);
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      const uint32_t idesc = umma_idesc_bf16(bn);
      for (int it = 0; it < nkt; ++it) {
        const int s = it % stages;
        if (!mbar_wait(&full_bar[s], (it / stages) & 1, &abort_flag, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* st = smem + (size_t)s * stage_bytes;
        const uint64_t ahi = umma_desc_sw128(st), alo = umma_desc_sw128(st + TC_A_BYTES);
        const uint64_t bhi = umma_desc_sw128(st + 2 * TC_A_BYTES), blo = umma_desc_sw128(st + 2 * TC_A_BYTES + b_bytes);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
          umma_bf16(tmem, ahi + adv, bhi + adv, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          umma_bf16(tmem, ahi + adv, blo + adv, idesc, 1u);
          umma_bf16(tmem, alo + adv, bhi + adv, idesc, 1u);
        }
        umma_commit(&empty_bar[s]);  // stage free once these MMAs have read it
      }
      umma_commit(&done_bar);  // accumulator complete (or nothing in flight after an abort)
    }
    __syncwarp();
    // epilogue: every warp reads its 32 TMEM lanes (rows)
    bool ok = mbar_wait(&done_bar, 0, &abort_flag, lim);
    // after an abort the MMAs already issued may still run: done_bar tracks
    // them all (the issuer commits it on every exit path)
    if (!ok) drained &= mbar_drain(&done_bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !abort_flag) {
      const int row = m0 + warp * 32 + lane;
      for (int c = 0; c < bn; c += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
        tmem_ld32(taddr, r);
        tmem_ld_wait();
        if (row < P.M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c + j;
            if (col >= P.N) break;
            const float v = __uint_as_float(r[j]);
            if (P.splits == 1)
              P.out[(size_t)row + (size_t)col * P.ldo] = P.alpha * (double)v;
            else
              P.part[((size_t)split * P.N + col) * P.M + row] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  // every thread is past its drain: nothing of this CTA is in flight (or a
  // drain itself gave up, reported as error 2)
  const int undrained = __syncthreads_or(drained ? 0 : 1);
  if (threadIdx.x == 0 && (abort_flag || undrained)) atomicMax(P.err, undrained ? 2 : 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// out[:, col] = alpha * sum_s part[s][:, col]  (FP64, column-major)
__global__ void k_tc_reduce(const float* part, int splits, int M, int N, double alpha, double* out, int ldo) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)M * N) return;
  int row = (int)(t % M), col = (int)(t / M);
  double s = 0.0;
  for (int k = 0; k < splits; ++k) s += (double)part[((size_t)k * N + col) * M + row];
  out[(size_t)row + (size_t)col * ldo] = alpha * s;
}

// hi = rn_bf16(x), lo = rn_bf16(x - hi) for a rows x cols FP64 block
__global__ void k_split_bf16(const double* src, int lds, int rows, int cols, __nv_bfloat16* hi, __nv_bfloat16* lo,
                             int ldd) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)rows * cols) return;
  int i = (int)(t % rows), j = (int)(t / rows);
  double x = src[(size_t)i + (size_t)j * lds];
  __nv_bfloat16 h = __float2bfloat16_rn((float)x);
  __nv_bfloat16 l = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
  hi[(size_t)i + (size_t)j * ldd] = h;
  lo[(size_t)i + (size_t)j * ldd] = l;
}

}  // namespace sdpg

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace sdpg {

// bf16 matrix viewed as `rows` rows of `inner` contiguous elements, row
// stride ld elements; box = 64 (inner) x box_rows, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const void* base, int inner, int rows, int ld, int box_rows) {
  return tc::make_map_bf16(map, base, inner, rows, ld, 1, box_rows);
}

// out (n x N, FP64, ld ldo) = alpha * W B with W given as bf16 hi/lo (n x n,
// ld ldw) and B as bf16 hi/lo (n x N, ld ldb).  part: FP32 workspace of
// at least 8 * n * N floats.  Returns 0, or -1 if the tensor maps could not
// be built (nothing launched).
int tc_wprod(cudaStream_t s, const void* whi, const void* wlo, int ldw, const void* bhi, const void* blo, int ldb,
             int n, int N, double alpha, double* out, int ldo, float* part, int* err, int num_sms,
             unsigned long long limit_ns) {
  if (n < 1 || N < 1) return 0;
  int bn = ((N + 15) / 16) * 16;
  if (bn > 256) bn = 256;
  const int ntn = (N + bn - 1) / bn;
  const int ntm = (n + TC_BM - 1) / TC_BM;
  const int kt = (n + TC_BK - 1) / TC_BK;
  int splits = 1;
  while (splits < 8 && ntm * ntn * splits * 2 <= num_sms && kt / (splits * 2) >= 4) splits *= 2;
  const int per = (kt + splits - 1) / splits;
  splits = (kt + per - 1) / per;
  const int stage_bytes = 2 * TC_A_BYTES + 2 * bn * TC_BK * 2;
  int stages = (220 * 1024) / stage_bytes;
  if (stages > 4) stages = 4;
  if (stages < 2) stages = 2;
  CUtensorMap mwh, mwl, mbh, mbl;
  if (!make_map(&mwh, whi, n, n, ldw, TC_BM) || !make_map(&mwl, wlo, n, n, ldw, TC_BM) ||
      !make_map(&mbh, bhi, n, N, ldb, bn) || !make_map(&mbl, blo, n, N, ldb, bn))
    return -1;
  TcParams P;
  P.M = n;
  P.N = N;
  P.K = n;
  P.splits = splits;
  P.ktiles_per = per;
  P.bn = bn;
  P.stages = stages;
  P.alpha = alpha;
  P.out = out;
  P.ldo = ldo;
  P.part = part;
  P.err = err;
  P.limit_ns = limit_ns;
  const size_t smem = (size_t)stages * stage_bytes + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_wprod, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
    attr = true;
  }
  k_tc_wprod<<<dim3(ntm, ntn, splits), 128, smem, s>>>(mwh, mwl, mbh, mbl, P);
  if (splits > 1) {
    long tot = (long)n * N;
    k_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, splits, n, N, alpha, out, ldo);
  }
  return 0;
}

void split_bf16(cudaStream_t s, const double* src, int lds, int rows, int cols, void* hi, void* lo, int ldd) {
  long tot = (long)rows * cols;
  if (tot <= 0) return;
  k_split_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, rows, cols, (__nv_bfloat16*)hi,
                                                            (__nv_bfloat16*)lo, ldd);
}

}  // namespace sdpg
