// admm_kernels.cu -- the ADMM steps of Algorithm 1 around the projection:
// the linear step (Eq. kkt_system) with its Woodbury/block elimination, the
// relaxation and the dual update, and the termination/infeasibility
// reductions of Section 5.
//
// The problem is min <C,X> s.t. A(X) = b, X psd, in form (P) with P = 0,
// q = C, A-bar = [A; I] and cone {b} x S+.  With s = sigma + rho and
// t = z_e - y_e/rho, one iteration is
//   r  = sigma x - C + rho Z - Y + rho A^T(t)
//   x~ = (r - rho A^T(v)) / s,     v = K^{-1} A(r),  K = s I + rho A A^T
//   W  = alpha x~ + (1-alpha) Z + Y/rho,   x <- alpha x~ + (1-alpha) x
//   y_e <- rho (alpha A(x~) + (1-alpha) z_e + y_e/rho - b),  z_e <- b
// (A(x~) = v exactly, since K v = A(r)), followed by Z = Pi(W) and
// Y = rho (W - Z) in the projection kernels.
//
// The dense n x n part is one elementwise pass (k_admm_dense) that ignores
// A; the sparse terms A^T(t) and A^T(v) live only on the positions A
// touches and are added by k_admm_sparse_fix.
#include "common.cuh"
#include "kernels.h"

namespace sdpg {

// r on the sparse positions (needed for u = A(r)).
__global__ void k_admm_sparse_r(Inst* insts, WorkMap wm) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int e = local * blockDim.x + threadIdx.x;
  if (e >= I.nent) return;
  int i = I.ent_i[e], j = I.ent_j[e];
  size_t q = idx2(i, j, I.ld);
  double r = I.sigma * I.x[q] - I.C[q] + I.rho * I.Z[q] - I.Y[q];
  double acc = 0.0;
  for (int k = I.ent_ptr[e]; k < I.ent_ptr[e + 1]; ++k) {
    int c = I.ent_con[k];
    acc += I.ent_val[k] * (I.ze[c] - I.ye[c] / I.rho);
  }
  I.ent_r[e] = r + I.rho * acc;
}

// u = A(r): u_p = sum over the entries of A_p of weight * r
__global__ void k_admm_cons_u(Inst* insts, WorkMap wm) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int p = local * blockDim.x + threadIdx.x;
  if (p >= I.mc) return;
  double acc = 0.0;
  for (int k = I.con_ptr[p]; k < I.con_ptr[p + 1]; ++k) acc += I.con_w[k] * I.ent_r[I.con_ent[k]];
  I.u[p] = acc;
}

// v = K^{-1} u by block elimination (one CTA per instance), then the
// equality-block dual update.  snapshot: keep y_e before the update.
__global__ void k_admm_ksolve(Inst* insts, const int* list) {
  const Inst& I = insts[list[blockIdx.x]];
  const int snapshot = I.ctl->snap;
  const int mc = I.mc, nF = I.nF;
  double* v = I.v;
  // F rows: t_f = u_f - sum_d K_fd u_d / K_dd  (stored in v[f] temporarily)
  for (int a = threadIdx.x; a < nF; a += blockDim.x) {
    int f = I.Flist[a];
    double acc = I.u[f];
    for (int k = I.k_ptr[f]; k < I.k_ptr[f + 1]; ++k) {
      int d = I.k_col[k];
      if (I.isD[d]) acc -= I.k_val[k] * I.u[d] / I.kdiag[d];
    }
    v[f] = acc;
  }
  __syncthreads();
  // Schur solve S v_F = t_F with S = Lf Lf^T (forward, then backward)
  __shared__ double red[32];
  for (int i = 0; i < nF; ++i) {
    double part = 0.0;
    for (int k = threadIdx.x; k < i; k += blockDim.x) part += I.Lf[idx2(i, k, nF)] * v[I.Flist[k]];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      int f = I.Flist[i];
      v[f] = (v[f] - s) / I.Lf[idx2(i, i, nF)];
    }
    __syncthreads();
  }
  for (int i = nF - 1; i >= 0; --i) {
    double part = 0.0;
    for (int k = i + 1 + threadIdx.x; k < nF; k += blockDim.x) part += I.Lf[idx2(k, i, nF)] * v[I.Flist[k]];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      int f = I.Flist[i];
      v[f] = (v[f] - s) / I.Lf[idx2(i, i, nF)];
    }
    __syncthreads();
  }
  // D rows: v_d = (u_d - sum_f K_df v_f) / K_dd
  for (int d = threadIdx.x; d < mc; d += blockDim.x) {
    if (!I.isD[d]) continue;
    double acc = I.u[d];
    for (int k = I.k_ptr[d]; k < I.k_ptr[d + 1]; ++k) {
      int f = I.k_col[k];
      if (!I.isD[f]) acc -= I.k_val[k] * v[f];
    }
    v[d] = acc / I.kdiag[d];
  }
  __syncthreads();
  // tv = t - v; y_e <- rho(alpha v + (1-alpha) z_e + y_e/rho - b); z_e <- b
  const double rho = I.rho, alpha = I.alpha;
  for (int p = threadIdx.x; p < mc; p += blockDim.x) {
    double ye = I.ye[p], ze = I.ze[p];
    I.tv[p] = (ze - ye / rho) - v[p];
    if (snapshot) I.yeprev[p] = ye;
    double we = alpha * v[p] + (1.0 - alpha) * ze + ye / rho;
    I.ye[p] = rho * (we - I.b[p]);
    I.ze[p] = I.b[p];
  }
}

// sparse correction of x~: (rho/s) A^T(t - v) on the sparse positions
__global__ void k_admm_sparse_corr(Inst* insts, WorkMap wm) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int e = local * blockDim.x + threadIdx.x;
  if (e >= I.nent) return;
  double acc = 0.0;
  for (int k = I.ent_ptr[e]; k < I.ent_ptr[e + 1]; ++k) acc += I.ent_val[k] * I.tv[I.ent_con[k]];
  I.ent_corr[e] = I.rho / (I.sigma + I.rho) * acc;
}

// Dense elementwise part: x~ = (sigma x - C + rho Z - Y)/s,
// W = alpha x~ + (1-alpha) Z + Y/rho, x <- alpha x~ + (1-alpha) x.
// snapshot: keep x and Y before the update (for delta x, delta y).
// Also writes the split-BF16 operands of W when the instance needs them.
__global__ void k_admm_dense(Inst* insts, WorkMap wm) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const int snapshot = I.ctl->snap;
  const size_t total = (size_t)I.ld * I.n;
  const double rho = I.rho, sigma = I.sigma, alpha = I.alpha, s = sigma + rho;
  for (size_t q = (size_t)local * blockDim.x * 4 + threadIdx.x; q < total && q < (size_t)(local + 1) * blockDim.x * 4;
       q += blockDim.x) {
    int i = (int)(q % I.ld);
    if (i >= I.n) continue;
    double x = I.x[q], Z = I.Z[q], Y = I.Y[q], C = I.C[q];
    if (snapshot) {
      I.xprev[q] = x;
      I.Yprev[q] = Y;
    }
    double xt = (sigma * x - C + rho * Z - Y) / s;
    I.W[q] = alpha * xt + (1.0 - alpha) * Z + Y / rho;
    I.x[q] = alpha * xt + (1.0 - alpha) * x;
  }
}

__global__ void k_admm_sparse_fix(Inst* insts, WorkMap wm) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int e = local * blockDim.x + threadIdx.x;
  if (e >= I.nent) return;
  int i = I.ent_i[e], j = I.ent_j[e];
  double d = I.alpha * I.ent_corr[e];
  size_t q = idx2(i, j, I.ld);
  I.W[q] += d;
  I.x[q] += d;
  if (i != j) {
    size_t qt = idx2(j, i, I.ld);
    I.W[qt] += d;
    I.x[qt] += d;
  }
}

// ---------------------------------------------------------------------------
// Termination and infeasibility reductions (Section 5 and Section 5.2).
// The Check struct of each instance must be zeroed before these run.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;  // valid in thread 0
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, sh[w]);
  return s;
}

__global__ void k_check_dense(Inst* insts, WorkMap wm) {
  __shared__ double sh[32];
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const size_t total = (size_t)I.ld * I.n;
  double rp = 0, rd = 0, nx = 0, nz = 0, nC = 0, nY = 0, obj = 0, ndY = 0, atd = 0, ndx = 0, cdx = 0;
  for (size_t q = (size_t)local * blockDim.x * 4 + threadIdx.x; q < total && q < (size_t)(local + 1) * blockDim.x * 4;
       q += blockDim.x) {
    int i = (int)(q % I.ld);
    if (i >= I.n) continue;
    double x = I.x[q], Z = I.Z[q], Y = I.Y[q], C = I.C[q], xp = I.xprev[q], Yp = I.Yprev[q];
    bool sp = (I.smask[q >> 5] >> (q & 31)) & 1u;
    rp = fmax(rp, fabs(x - Z));
    nx = fmax(nx, fabs(x));
    nz = fmax(nz, fabs(Z));
    nC = fmax(nC, fabs(C));
    nY = fmax(nY, fabs(Y));
    obj += C * x;
    ndY = fmax(ndY, fabs(Y - Yp));
    ndx = fmax(ndx, fabs(x - xp));
    cdx += C * (x - xp);
    if (!sp) {
      rd = fmax(rd, fabs(C + Y));
      atd = fmax(atd, fabs(Y - Yp));
    }
  }
  Check* K = I.chk;
  double v;
  v = block_max(rp, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->rp_dense, v);
  v = block_max(rd, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->rd_dense, v);
  v = block_max(nx, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nx, v);
  v = block_max(nz, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nz, v);
  v = block_max(nC, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nC, v);
  v = block_max(nY, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nY, v);
  v = block_max(ndY, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->ndY, v);
  v = block_max(atd, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->at_dense, v);
  v = block_max(ndx, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->ndx, v);
  v = block_sum(obj, sh); if (threadIdx.x == 0) atomicAdd(&K->obj, v);
  v = block_sum(cdx, sh); if (threadIdx.x == 0) atomicAdd(&K->cdx, v);
}

// On the sparse positions: C + Y + A^T y and dY + A^T dy.
__global__ void k_check_sparse(Inst* insts, WorkMap wm) {
  __shared__ double sh[32];
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int e = local * blockDim.x + threadIdx.x;
  double rd = 0, at = 0, naty = 0;
  if (e < I.nent) {
    size_t q = idx2(I.ent_i[e], I.ent_j[e], I.ld);
    double aty = 0, atdy = 0;
    for (int k = I.ent_ptr[e]; k < I.ent_ptr[e + 1]; ++k) {
      int c = I.ent_con[k];
      aty += I.ent_val[k] * I.ye[c];
      atdy += I.ent_val[k] * (I.ye[c] - I.yeprev[c]);
    }
    rd = fabs(I.C[q] + I.Y[q] + aty);
    at = fabs(I.Y[q] - I.Yprev[q] + atdy);
    naty = fabs(I.Y[q] + aty);
  }
  Check* K = I.chk;
  double v;
  v = block_max(rd, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->rd_sparse, v);
  v = block_max(at, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->at_sparse, v);
  v = block_max(naty, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nATy, v);
}

// Per constraint: A(x) - b, A(dx), dy_e, b^T dy.
__global__ void k_check_cons(Inst* insts, WorkMap wm) {
  __shared__ double sh[32];
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  int p = local * blockDim.x + threadIdx.x;
  double rpc = 0, nax = 0, ndy = 0, bdy = 0, adx = 0;
  if (p < I.mc) {
    double ax = 0, adxv = 0;
    for (int k = I.con_ptr[p]; k < I.con_ptr[p + 1]; ++k) {
      int e = I.con_ent[k];
      size_t q = idx2(I.ent_i[e], I.ent_j[e], I.ld);
      ax += I.con_w[k] * I.x[q];
      adxv += I.con_w[k] * (I.x[q] - I.xprev[q]);
    }
    rpc = fabs(ax - I.b[p]);
    nax = fabs(ax);
    double dy = I.ye[p] - I.yeprev[p];
    ndy = fabs(dy);
    bdy = I.b[p] * dy;
    adx = fabs(adxv);
  }
  Check* K = I.chk;
  double v;
  v = block_max(rpc, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->rp_cons, v);
  v = block_max(nax, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->nAx, v);
  v = block_max(ndy, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->ndy_e, v);
  v = block_max(adx, sh); if (threadIdx.x == 0) atomic_max_nonneg(&K->adx, v);
  v = block_sum(bdy, sh); if (threadIdx.x == 0) atomicAdd(&K->bdy, v);
}

// Cone membership by Cholesky (Section 5 footnote): E <- sgn*(M - Mprev)/scale
// + shift*I, then an in-place Cholesky in one CTA; ctl->chol_fail = 0 when
// positive definite.  `which` 0: M = Y (primal certificate, sgn = -1),
// 1: M = x (dual certificate, sgn = +1).
__global__ void k_cone_fill(Inst* insts, WorkMap wm, const double* scale, int which, double shift) {
  int local;
  int ii = find_inst(wm, blockIdx.x, &local);
  const Inst& I = insts[ii];
  const size_t total = (size_t)I.ld * I.n;
  double sc = scale[ii];
  for (size_t q = (size_t)local * blockDim.x * 4 + threadIdx.x; q < total && q < (size_t)(local + 1) * blockDim.x * 4;
       q += blockDim.x) {
    int i = (int)(q % I.ld), j = (int)(q / I.ld);
    double d = which == 0 ? -(I.Y[q] - I.Yprev[q]) / sc : (I.x[q] - I.xprev[q]) / sc;
    I.E[q] = d + (i == j ? shift : 0.0);
  }
}

__global__ void k_cone_chol(Inst* insts, const int* list) {
  const Inst& I = insts[list[blockIdx.x]];
  const int n = I.n, ld = I.ld;
  double* A = I.E;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = A[idx2(j, j, ld)];
      if (!(d > 0.0)) fail = j + 1;
      else A[idx2(j, j, ld)] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    double ljj = A[idx2(j, j, ld)];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[idx2(i, j, ld)] /= ljj;
    __syncthreads();
    int w = n - j - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      int r = t % w, c = t / w;
      if (r < c) continue;
      int i = j + 1 + r, k = j + 1 + c;
      A[idx2(i, k, ld)] -= A[idx2(i, j, ld)] * A[idx2(k, j, ld)];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) I.ctl->chol_fail = fail;
}

}  // namespace sdpg
