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

namespace sdpg {

static constexpr int TC_BM = 128;
static constexpr int TC_BK = 64;                       // bf16 elements per 128-byte row
static constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;   // 16 KiB

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false when `limit_ns` of elapsed time passed (the wait then
// raises the CTA's abort flag) or another thread of the CTA aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
// clean-up wait after an abort: ignores the abort flag
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer_ns() - t0 > kDrainLimitNs) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// K-major operand tile, rows of 128 bytes, 8-row swizzle atoms 1024 B apart
__device__ __forceinline__ uint64_t umma_desc_sw128(const void* tile) {
  uint64_t addr = smem_u32(tile);
  uint64_t d = (addr & 0x3FFFFull) >> 4;  // start address
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                 // layout: 128-byte swizzle
  return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// D (128 x BN, FP32 in TMEM) += op over K; bf16 inputs, K-major A and B
__host__ __device__ __forceinline__ uint32_t umma_idesc_bf16(int bn) {
  return (1u << 4)                      // D format: F32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(bn >> 3) << 17)  // N / 8
         | ((uint32_t)(TC_BM >> 4) << 24);  // M / 16
}

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
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
            "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// bf16 matrix viewed as `rows` rows of `inner` contiguous elements, row
// stride ld elements; box = 64 (inner) x box_rows, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const void* base, int inner, int rows, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) || ((ld * 2) & 15)) return false;  // TMA needs 16-byte alignment
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
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
