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

// The harmonic Ritz matrix of an augmented GCRO-DR cycle (dense.cuh harmonic_matrix): G = [[I_k, B],
// [0, Hbar]] with Hbar (j+1) x j and B k x j (both row-major, interleaved), S = [[Stop, 0],
// [Sbot, I]]; Hbar is reduced by Givens rotations exactly as the solver's per-step finalize does,
// B is handed over with leading dimension ld_b >= k (as the solver stores it).  Returns the k+j
// eigenvalues nu of M = R_G^{-1} (Q_G^H S) in nu (2*(k+j) doubles).
int host_harmonic_nu(int k, int j, int ld_b, const double* hbar, const double* b, const double* stop,
                     const double* sbot, double* nu) {
  const int n = k + j, ldh = j + 1, ld = n + 1;
  std::vector<cd> R(ldh * j), Bc(ld_b * (j > 0 ? j : 1), mk(0.0, 0.0)), col(j + 2), sn(j), M(ld * ld);
  std::vector<double> cs(j);
  const cd* H = reinterpret_cast<const cd*>(hbar);
  for (int c = 0; c < j; ++c) {
    for (int i = 0; i <= c + 1; ++i) col[i] = H[i * j + c];
    for (int i = 0; i < c; ++i) {
      const cd u = col[i], w = col[i + 1];
      col[i] = add(scal(u, cs[i]), mul(sn[i], w));
      col[i + 1] = sub(scal(w, cs[i]), conjmul(sn[i], u));
    }
    double cc;
    cd sg, r;
    givens(col[c], col[c + 1], cc, sg, r);
    cs[c] = cc;
    sn[c] = sg;
    col[c] = r;
    for (int i = 0; i <= c; ++i) R[c * ldh + i] = col[i];
  }
  const cd* Bi = reinterpret_cast<const cd*>(b);
  for (int c = 0; c < j; ++c)
    for (int i = 0; i < k; ++i) Bc[c * ld_b + i] = Bi[i * j + c];
  HostTeam tm;
  int rc = harmonic_matrix(tm, k, j, cs.data(), sn.data(), R.data(), ldh, Bc.data(), ld_b,
                           reinterpret_cast<const cd*>(stop), reinterpret_cast<const cd*>(sbot), M.data(), ld);
  if (rc) return rc;
  std::vector<cd> A(n * n), Z(n * n), v(n);
  std::vector<double> sc(8);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < n; ++c) {
      A[i * n + c] = M[i * ld + c];
      Z[i * n + c] = mk(i == c ? 1.0 : 0.0, 0.0);
    }
  hessenberg(tm, A.data(), Z.data(), n, n, v.data(), sc.data());
  rc = schur_qr(tm, A.data(), Z.data(), n, n, false);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    nu[2 * i] = A[i * n + i].x;
    nu[2 * i + 1] = A[i * n + i].y;
  }
  return 0;
}

}  // extern "C"
