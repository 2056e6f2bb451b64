// runtime.h -- host-side set-up structures of libsdpgpu.
#pragma once
#include <vector>

namespace sdpg {

// Sparse operators of one instance and the block factorisation of
// K = (sigma+rho) I + rho A A^T used by the linear step of Algorithm 1.
struct HostSetup {
  int nent = 0;                       // distinct positions (i <= j) touched by A
  std::vector<int> ent_i, ent_j;      // nent
  std::vector<int> ent_ptr;           // nent+1: entry -> its (constraint, value) list
  std::vector<int> ent_con;
  std::vector<double> ent_val;
  std::vector<int> con_ptr;           // m+1: constraint -> its (entry, weight) list
  std::vector<int> con_ent;
  std::vector<double> con_w;          // value * (i == j ? 1 : 2)
  std::vector<double> kdiag;          // K_pp
  std::vector<int> isD, fpos, Flist;  // D: independent set (diagonal block), F: the rest
  std::vector<int> k_ptr, k_col;      // off-diagonal K entries, CSR by row
  std::vector<double> k_val;
  int nF = 0;
  std::vector<double> Lf;             // nF x nF Cholesky factor of the Schur complement
};

// Returns 0 (SDP_OK) or a negative sdp_status.
int host_setup(int n, int m, long nnz, const int* cp, const int* ci, const int* cj, const double* cv, double sigma,
               double rho, HostSetup* out);

}  // namespace sdpg
