// Host build of device helpers of the library, for CPU tests of their
// arithmetic: the two Sturm counts and inverse iteration of the Rayleigh-Ritz
// eigensolvers (paper_1912_02767_gb300/csrc/tri_common.cuh) and the Philox
// generator of the expansion columns (csrc/common.cuh).  Test
// infrastructure only; nothing here runs on a GPU.
#include "../../paper_1912_02767_gb300/csrc/tri_common.cuh"

using namespace sdpg::tri;

extern "C" {
// eigenvalues of the tridiagonal (d, e2 = e^2) below x, by the signs of the
// leading principal minors
int h_count_minors(const double* d, const double* e2, int p, double x) { return sturm_below_minors(d, e2, p, x); }
// the same by the pivots of LDL^T (pivots below pivmin taken as -pivmin)
int h_count_ratio(const double* d, const double* e2, int p, double x, double pivmin) {
  return sturm_below(d, e2, p, x, pivmin);
}
// inverse iteration for the eigenvector nearest the shift sg; z (p) out,
// w (3 p) scratch; q selects the start vector
void h_inv_iter(const double* d, const double* e, int p, double sg, double* z, double* w, int q) {
  inv_iter<double, double>(d, e, p, sg, z, 1, w, 1, q);
}
// one Philox4x32-10 block: ctr (4 words) in, out (4 words)
void h_philox(const unsigned* ctr, unsigned k0, unsigned k1, unsigned* out) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  sdpg::philox4x32_10(c, k0, k1);
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}
}
