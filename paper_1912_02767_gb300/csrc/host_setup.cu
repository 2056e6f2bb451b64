// host_setup.cu -- one-time set-up of an instance on the host: the sparse
// operator structures (position-major and constraint-major) and the
// factorisation of K = (sigma+rho) I_m + rho A A^T that the linear step of
// Algorithm 1 solves with every iteration (the paper factors its KKT
// matrix once and substitutes each iteration, Section 5).
//
// K is eliminated by blocks: D is an independent set of the graph of
// A A^T (so K_DD is diagonal), F the remaining constraints, and the dense
// Schur complement K_FF - K_FD K_DD^{-1} K_DF is factored by Cholesky.
// For max-cut and Lovasz-theta constraints A A^T is diagonal (F empty);
// diag(X) = 1 plus a trace row gives |F| = 1.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "../../include/sdpgpu.h"
#include "runtime.h"

namespace sdpg {

static const int kMaxSchur = 4096;

int host_setup(int n, int m, long nnz, const int* cp, const int* ci, const int* cj, const double* cv, double sigma,
               double rho, HostSetup* H) {
  const double s = sigma + rho;
  // positions: key = i * n + j (i <= j)
  std::vector<long> order(nnz);
  std::iota(order.begin(), order.end(), 0L);
  std::sort(order.begin(), order.end(), [&](long a, long b) {
    long ka = (long)ci[a] * n + cj[a], kb = (long)ci[b] * n + cj[b];
    if (ka != kb) return ka < kb;
    return a < b;
  });
  H->ent_ptr.assign(1, 0);
  std::vector<int> ent_of(nnz);
  for (long t = 0; t < nnz; ++t) {
    long q = order[t];
    bool fresh = (t == 0) || ci[q] != ci[order[t - 1]] || cj[q] != cj[order[t - 1]];
    if (fresh) {
      H->ent_i.push_back(ci[q]);
      H->ent_j.push_back(cj[q]);
      if (t) H->ent_ptr.push_back((int)t);
    }
    H->ent_con.push_back(cp[q]);
    H->ent_val.push_back(cv[q]);
    ent_of[q] = (int)H->ent_i.size() - 1;
  }
  H->nent = (int)H->ent_i.size();
  H->ent_ptr.push_back((int)nnz);
  if (H->nent == 0) H->ent_ptr.assign(1, 0);
  // constraint-major lists
  H->con_ptr.assign(m + 1, 0);
  for (long t = 0; t < nnz; ++t) H->con_ptr[cp[t] + 1]++;
  for (int p = 0; p < m; ++p) H->con_ptr[p + 1] += H->con_ptr[p];
  H->con_ent.assign(nnz, 0);
  H->con_w.assign(nnz, 0.0);
  {
    std::vector<int> fill(H->con_ptr.begin(), H->con_ptr.end() - 1);
    for (long t = 0; t < nnz; ++t) {
      int p = cp[t], k = fill[p]++;
      H->con_ent[k] = ent_of[t];
      H->con_w[k] = cv[t] * (ci[t] == cj[t] ? 1.0 : 2.0);
    }
  }
  // A A^T: sum over positions of products of the constraint values there
  std::vector<std::unordered_map<int, double>> rows(m);
  for (int e = 0; e < H->nent; ++e) {
    double w = (H->ent_i[e] == H->ent_j[e]) ? 1.0 : 2.0;
    for (int a = H->ent_ptr[e]; a < H->ent_ptr[e + 1]; ++a)
      for (int b = H->ent_ptr[e]; b < H->ent_ptr[e + 1]; ++b)
        rows[H->ent_con[a]][H->ent_con[b]] += w * H->ent_val[a] * H->ent_val[b];
  }
  H->kdiag.assign(m, s);
  std::vector<int> degree(m, 0);
  for (int p = 0; p < m; ++p)
    for (auto& kv : rows[p]) {
      if (kv.first == p) H->kdiag[p] += rho * kv.second;
      else if (kv.second != 0.0) degree[p]++;
    }
  // independent set D, lowest degree first
  std::vector<int> byDeg(m);
  std::iota(byDeg.begin(), byDeg.end(), 0);
  std::stable_sort(byDeg.begin(), byDeg.end(), [&](int a, int b) { return degree[a] < degree[b]; });
  H->isD.assign(m, 0);
  for (int p : byDeg) {
    bool ok = true;
    for (auto& kv : rows[p])
      if (kv.first != p && kv.second != 0.0 && H->isD[kv.first]) { ok = false; break; }
    H->isD[p] = ok ? 1 : 0;
  }
  H->fpos.assign(m, -1);
  H->nF = 0;
  for (int p = 0; p < m; ++p)
    if (!H->isD[p]) { H->fpos[p] = H->nF++; H->Flist.push_back(p); }
  if (H->nF > kMaxSchur) return SDP_E_INVALID;
  // off-diagonal CSR (sorted columns for determinism)
  H->k_ptr.assign(m + 1, 0);
  for (int p = 0; p < m; ++p) {
    std::vector<std::pair<int, double>> ent;
    for (auto& kv : rows[p])
      if (kv.first != p && kv.second != 0.0) ent.push_back({kv.first, rho * kv.second});
    std::sort(ent.begin(), ent.end());
    for (auto& e2 : ent) { H->k_col.push_back(e2.first); H->k_val.push_back(e2.second); }
    H->k_ptr[p + 1] = (int)H->k_col.size();
  }
  // Schur complement and its Cholesky factor
  const int nF = H->nF;
  std::vector<double> S((size_t)nF * nF, 0.0);
  for (int a = 0; a < nF; ++a) {
    int f = H->Flist[a];
    S[a + (size_t)a * nF] = H->kdiag[f];
    for (int k = H->k_ptr[f]; k < H->k_ptr[f + 1]; ++k) {
      int q = H->k_col[k];
      if (!H->isD[q]) S[a + (size_t)H->fpos[q] * nF] += H->k_val[k];
    }
  }
  for (int d = 0; d < m; ++d) {
    if (!H->isD[d]) continue;
    for (int k1 = H->k_ptr[d]; k1 < H->k_ptr[d + 1]; ++k1)
      for (int k2 = H->k_ptr[d]; k2 < H->k_ptr[d + 1]; ++k2) {
        int a = H->fpos[H->k_col[k1]], b = H->fpos[H->k_col[k2]];
        S[a + (size_t)b * nF] -= H->k_val[k1] * H->k_val[k2] / H->kdiag[d];
      }
  }
  H->Lf.assign((size_t)nF * nF, 0.0);
  for (int j = 0; j < nF; ++j) {
    double d = S[j + (size_t)j * nF];
    for (int k = 0; k < j; ++k) d -= H->Lf[j + (size_t)k * nF] * H->Lf[j + (size_t)k * nF];
    if (!(d > 0.0)) return SDP_E_NUMERICAL;
    double l = sqrt(d);
    H->Lf[j + (size_t)j * nF] = l;
    for (int i = j + 1; i < nF; ++i) {
      double acc = S[i + (size_t)j * nF];
      for (int k = 0; k < j; ++k) acc -= H->Lf[i + (size_t)k * nF] * H->Lf[j + (size_t)k * nF];
      H->Lf[i + (size_t)j * nF] = acc / l;
    }
  }
  return SDP_OK;
}

}  // namespace sdpg
