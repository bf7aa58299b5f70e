// Host build of the library's small dense FP64 routines (single-lane team),
// used only by tests/test_dense_host.py to check them against LAPACK.
#include <cuda_runtime.h>  // double2
#include <cmath>
#include <cstring>
#include <vector>
#define DENSE_HD
#include "../paper_2205_09104_gb300/csrc/dense.cuh"

using namespace coarse::dense;

extern "C" {

// Eigen-decomposition of a dense complex m x m matrix (row-major, interleaved).
// lam: 2*m doubles; vecs: 2*m*m doubles, column q = eigenvector of lam[q] (unnormalised).
int host_eig(int m, const double* a, double* lam, double* vecs) {
  const int ld = m;
  std::vector<cd> A(m * m), Z(m * m), Y(m * m), v(m);
  std::vector<double> sc(8);
  std::memcpy(A.data(), a, sizeof(cd) * m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Z[i * ld + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  HostTeam tm;
  hessenberg(tm, A.data(), Z.data(), m, ld, v.data(), sc.data());
  int rc = schur_qr(tm, A.data(), Z.data(), m, ld, true);
  if (rc) return rc;
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  tri_eigvecs(tm, A.data(), m, ld, idx.data(), m, Y.data(), m);
  for (int i = 0; i < m; ++i) {
    lam[2 * i] = A[i * ld + i].x;
    lam[2 * i + 1] = A[i * ld + i].y;
  }
  for (int i = 0; i < m; ++i)
    for (int q = 0; q < m; ++q) {
      cd s = mk(0.0, 0.0);
      for (int l = 0; l < m; ++l) s = add(s, mul(Z[i * ld + l], Y[l * m + q]));
      vecs[2 * (i * m + q)] = s.x;
      vecs[2 * (i * m + q) + 1] = s.y;
    }
  return 0;
}

// Hessenberg form only: returns H and Z with A = Z H Z^H.
void host_hessenberg(int m, const double* a, double* h, double* z) {
  std::vector<cd> A(m * m), Z(m * m), v(m);
  std::vector<double> sc(8);
  std::memcpy(A.data(), a, sizeof(cd) * m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Z[i * m + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  HostTeam tm;
  hessenberg(tm, A.data(), Z.data(), m, m, v.data(), sc.data());
  std::memcpy(h, A.data(), sizeof(cd) * m * m);
  std::memcpy(z, Z.data(), sizeof(cd) * m * m);
}

void host_leja(int d, double* theta) {
  std::vector<cd> t(d), out(d);
  std::vector<int> used(d);
  std::memcpy(t.data(), theta, sizeof(cd) * d);
  leja_order(t.data(), d, used.data(), out.data());
  std::memcpy(theta, t.data(), sizeof(cd) * d);
}

void host_givens(const double* x, const double* y, double* out /* c, s.re, s.im, r.re, r.im */) {
  double c; cd s, r;
  givens(mk(x[0], x[1]), mk(y[0], y[1]), c, s, r);
  out[0] = c; out[1] = s.x; out[2] = s.y; out[3] = r.x; out[4] = r.y;
}

}  // extern "C"
