// kernels.h -- declarations of the sdpgpu device kernels and job records.
#pragma once
#include "common.cuh"

namespace sdpg {

enum { EPI_STORE = 0, EPI_PARTIAL = 1, EPI_RECON_POS = 2, EPI_RECON_NEG = 3 };

// One product of a batched GEMM launch (see k_gemm).
struct GemmJob {
  const double* A;
  const double* B;
  double* C;
  const double* colscale;  // optional scale of op(A)'s columns (the k index)
  const double* Eb;        // reconstruction: W
  double* C2;              // reconstruction: Y; Gram reduce: destination
  int lda, ldb, ldc;
  int M, N, K;
  int splits, tiles_m, tiles_n, epi;
  double alpha, beta, rho;
};

// admm_kernels.cu
__global__ void k_admm_sparse_r(Inst* insts, WorkMap wm);
__global__ void k_admm_cons_u(Inst* insts, WorkMap wm);
__global__ void k_admm_ksolve(Inst* insts, const int* list);
__global__ void k_admm_sparse_corr(Inst* insts, WorkMap wm);
__global__ void k_admm_dense(Inst* insts, WorkMap wm);
__global__ void k_admm_sparse_fix(Inst* insts, WorkMap wm);
__global__ void k_check_dense(Inst* insts, WorkMap wm);
__global__ void k_check_sparse(Inst* insts, WorkMap wm);
__global__ void k_check_cons(Inst* insts, WorkMap wm);
__global__ void k_cone_fill(Inst* insts, WorkMap wm, const double* scale, int which, double shift);
__global__ void k_cone_chol(Inst* insts, const int* list);

// lobpcg_kernels.cu
template <bool TA, bool TB, typename TC>
__global__ void k_gemm(const GemmJob* jobs, WorkMap wm);
__global__ void k_gram_reduce(const GemmJob* jobs, WorkMap wm, int symmetrize);
template <typename T>
__global__ void k_rr_smem(Inst* insts, const int* list, int u_global, int p_launch);
// largest trial subspace k_rr_smem<T> holds with both p x p workspaces in
// shared memory (2 p^2 elements of T <= 200 KiB), and with one of them
// (p^2 elements <= 205 KiB; the other in global memory)
constexpr int kRRSmemMaxF32 = 160;
constexpr int kRRSmemMaxF64 = 112;
constexpr int kRRSmem1MaxF32 = 224;
constexpr int kRRSmem1MaxF64 = 156;
constexpr int kRRGlobalMax = 1024;  // one-CTA Rayleigh-Ritz with both workspaces in global memory
// shared-memory bytes of k_rr_smem's rotation table + sort order for width p
__host__ __device__ inline size_t rr_table_bytes(int p, int tsize) {
  const int P2 = (p + 1) / 2;
  size_t b = (size_t)2 * P2 * tsize + (size_t)2 * P2 * sizeof(int) + (size_t)p * sizeof(int);
  return (b + 15) / 16 * 16;
}
// rr_tri.cu: Rayleigh-Ritz by tridiagonal reduction, one CTA (1024 threads)
// per instance; zsm = 1 keeps the p x keep Ritz block in shared memory
template <typename T>
__global__ void k_rr_tri(Inst* insts, const int* list, int zsm, unsigned smem_launch);
// dynamic shared memory of k_rr_tri<T> for width p, with the Ritz block of
// zk columns in shared memory (zk = keep) or in global memory (zk = 0)
__host__ __device__ inline size_t rr_tri_smem_bytes(int p, int zk, int tsize) {
  return ((size_t)p * (size_t)(p | 1) + 11 * (size_t)p + 1024 + (size_t)p * (size_t)zk) * (size_t)tsize;
}
constexpr size_t kRRTriSmemMax = 231936;  // 227 KiB per CTA less the kernel's static shared memory
// threads of a k_rr_tri CTA for widths up to p (p <= threads): fewer warps
// per barrier for narrow subspaces, all 32 for wide ones
constexpr int kRRTriMaxF64 = 1024;  // cap on the FP64 width of the one-CTA route (shared memory binds first)
inline int rr_tri_threads(int p) { return p <= 32 ? 128 : (p <= 64 ? 256 : (p <= 128 ? 512 : 1024)); }
__global__ void k_resid(Inst* insts, WorkMap wm);
__global__ void k_resid_finish(Inst* insts, const int* list, int last_allowed);
__global__ void k_compact(Inst* insts, WorkMap wm);
__global__ void k_fill_random(Inst* insts, WorkMap wm, const int* col0, const int* ncols, const int* draw,
                              const unsigned* stream, unsigned long long seed);

// rr_large.cu (cooperative, one matrix per launch)
template <typename T>
__global__ void k_chol_inv_coop(double* G, double* Linv, int p, double piv_min, GridBar* b);
template <typename T>
__global__ void k_jacobi_coop(double* H, double* H2, int ldh, double* U, int ldu, int p, double rel, double abs_eps,
                              int max_sweeps, const double* fro2, GridBar* b);
__global__ void k_diag_rank(const double* H, int ldh, int p, int* ord, int* fail);
__global__ void k_select_top(const double* H, int ldh, const double* U, int ldu, int p, int keep, const int* ord,
                             double* Usel, double* theta, int* npos);
__global__ void k_rr_large_finish(Ctl* ctl, const GridBar* b);

// rr_wide.cu (one wide subspace over the whole GPU, tridiagonal route)
template <typename T>
__global__ void k_trid_coop(const double* H, T* A, int p, int keep, double* vb, GridBar* b);
template <typename T>
__global__ void k_trid_tail(const T* A, int p, int keep, double* vb, GridBar* b);
constexpr int kLatrdNb = 64;   // panel width of the blocked tridiagonalization
constexpr int kLatrdOwn = 64;  // owned columns per CTA it can hold (grid >= p / 63)
__global__ void k_latrd_coop(double* A, int p, int keep, int j0, int j1, double* Vp, double* Wp, double* Kg,
                             double* pt, double* vb, GridBar* b);
__global__ void k_latrd_wfinal(const double* Vp, double* Wp, const double* Kg, int p, int r0, int nc);
__global__ void k_sym_copy(const double* H, double* A, int p);
// Householder tridiagonalization on one thread-block cluster (distributed
// shared memory); host side: cluster width for p (16, 8, or 0 = does not
// fit) and the launch (0 ok, -1 refused)
constexpr int kTridClThreads = 512;
constexpr size_t kTridClSmemMax = 230400;
__host__ __device__ inline size_t trid_cluster_smem(int p, int cl) {
  const int ncl = (p + cl - 1) / cl, ldl = p | 1;
  return ((size_t)ncl * ldl + 6 * (size_t)p + 8 + kTridClThreads + 32) * sizeof(double);
}
int trid_cluster_width(int p);
int trid_cluster_max_p(int cl);
int trid_cluster(cudaStream_t s, int cl, const double* H, double* A, int p, int keep, double* vb, GridBar* b);
template <typename TS, typename T>
__global__ void k_trid_eig(double* vb, int p, int keep, int S, int refine, int final, double* theta, int* npos,
                           const GridBar* b);
template <typename T>
__global__ void k_trid_shift(double* vb, int p, int keep, const GridBar* b);
template <typename T>
__global__ void k_trid_invit(double* vb, int p, int keep, double* Z, T* WS, const GridBar* b);
template <typename T>
__global__ void k_trid_backtr(const T* A, double* vb, int p, int keep, double* Y, int nv, const GridBar* b);
constexpr int kTridBacktrNv = 16;  // vectors per CTA of k_trid_backtr (at most)
// dynamic shared memory of k_trid_backtr: nv vectors, three reflector buffers, tau
inline size_t rr_backtr_smem_bytes(int p, int nv, int tsize) { return (size_t)(nv + 4) * p * tsize; }
constexpr size_t kBacktrSmemMax = 230400;  // 227 KiB per CTA less the kernel's static shared memory (<= 2 KiB)

// rr_blocked.cu (blocked Cholesky/inverse and compact-WY back-transform,
// their products on the tensor cores)
constexpr int kBlk = 128;  // diagonal block / reflector block width
constexpr size_t kBlkSmem = (size_t)kBlk * (kBlk + 1) * sizeof(double);
// diagonal block of the blocked Cholesky/inverse: narrower than kBlk, since
// its O(b^3) FP64 work runs on one SM while the panel and trailing products
// run on the tensor cores
constexpr int kPotrfBlk = 64;
constexpr size_t potrf_block_smem(int blk) { return (size_t)blk * (blk + 1) * sizeof(double); }
template <int BLK>
__global__ void k_potrf_inv_block(double* G, int ldg, double* Linv, int ldl, int j0, int bb, double piv_min,
                                  GridBar* bar);
__global__ void k_wy_vmat(const double* A, int p, int nref, double* V);
__global__ void k_wy_tmat(double* Tall, const double* tau, int nref);

// jacobi_kernels.cu (exact branch)
__global__ void k_jac_init(Inst* insts, WorkMap wm, int negate);
__global__ void k_jac_angles(Inst* insts, WorkMap wm, int round);
__global__ void k_jac_apply(Inst* insts, WorkMap wm, int round);
__global__ void k_jac_sort(Inst* insts, const int* list);
__global__ void k_jac_gather(Inst* insts, WorkMap wm);
__global__ void k_fro2(Inst* insts, WorkMap wm, int to_w);
__global__ void k_fro2_det(Inst* insts, const int* list);
__global__ void k_fro2_mat(const double* A, int ld, int rows, int cols, double* dst);
__global__ void k_seed_block(Inst* insts, WorkMap wm);
__global__ void k_copy_cols(const double* src, int lds, double* dst, int ldd, int rows, int cols, double scale);

// bj_eig.cu (host driver): block Jacobi, returns sweeps or -1
int block_jacobi(cudaStream_t s, double* H, int ldh, double* U, int ldu, int p, bool f32, double eps,
                 const double* fro2_dev, int max_sweeps, double* Q, double* offp, double* offh);

// tc_gemm.cu (host wrappers)
// *err: 0 untouched; 1 a bounded wait gave up; 2 a clean-up wait gave up too
int tc_wprod(cudaStream_t s, const void* whi, const void* wlo, int ldw, const void* bhi, const void* blo, int ldb,
             int n, int N, double alpha, double* out, int ldo, float* part, int* err, int num_sms,
             unsigned long long limit_ns);
void split_bf16(cudaStream_t s, const double* src, int lds, int rows, int cols, void* hi, void* lo, int ldd);

// oz_gemm.cu: C = alpha op(A) op(B) + beta C (FP64 column-major; op 'N' or
// 'T') to FP64 accuracy on the tensor cores; `work` holds oz_work_bytes.
// Returns 0, -1 (tensor maps / attributes refused, nothing launched) or -2
// (work too small).  *err as for tc_wprod.
size_t oz_work_bytes(int M, int N, int K);
void symmetrize(cudaStream_t s, double* X, int p, int ld);
int oz_gemm(cudaStream_t s, char ta, const double* A, int lda, char tb, const double* B, int ldb, int M, int N,
            int K, double alpha, double beta, double* C, int ldc, void* work, size_t work_bytes, int* err,
            int num_sms, unsigned long long limit_ns);

}  // namespace sdpg
