// Small dense FP64 complex linear algebra of the Krylov solver, written for a
// "team" of lanes that share the matrices in (shared) memory:
//   - on the device a team is one warp (32 lanes, __syncwarp);
//   - compiled for the host a team is a single lane (used only by the unit
//     tests, which check these routines against LAPACK on the CPU).
// Matrices are row-major with a fixed leading dimension.  Every lane reads
// the same control data after each sync, so scalar decisions are taken
// identically by all lanes; shared scalars are written by lane 0 only.
//
// Contents
//   givens        plane rotation [c s; -conj(s) c] zeroing the second entry
//   hessenberg    Householder reduction A = Z H Z^H
//   schur_qr      complex single-shift QR iteration (Wilkinson shift, deflation)
//                 to upper-triangular T, accumulating Z
//   tri_eigvecs   eigenvectors of T by back substitution
//   leja_order    Alg. 2 (Leja ordering) with the tie rule: larger score, then
//                 larger real part, larger imaginary part, lower index
#pragma once

#include <math.h>

#ifndef DENSE_HD
#define DENSE_HD __host__ __device__
#endif

namespace coarse {
namespace dense {

typedef double2 cd;

DENSE_HD inline cd mk(double r, double i) { cd z; z.x = r; z.y = i; return z; }
DENSE_HD inline cd add(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
DENSE_HD inline cd sub(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
DENSE_HD inline cd mul(cd a, cd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
DENSE_HD inline cd cmulc(cd a, cd b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a*conj(b)
DENSE_HD inline cd conjmul(cd a, cd b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); } // conj(a)*b
DENSE_HD inline cd conj(cd a) { return mk(a.x, -a.y); }
DENSE_HD inline cd scal(cd a, double s) { return mk(a.x * s, a.y * s); }
DENSE_HD inline double abs2(cd a) { return a.x * a.x + a.y * a.y; }
DENSE_HD inline double cabs(cd a) { return hypot(a.x, a.y); }
DENSE_HD inline cd cdiv(cd a, cd b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, den = b.x + b.y * r;
    return mk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  const double r = b.x / b.y, den = b.x * r + b.y;
  return mk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
DENSE_HD inline cd csqrt(cd z) {
  const double r = cabs(z);
  if (r == 0.0) return mk(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return mk(t, z.y / (2.0 * t));
  return mk(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}
DENSE_HD inline bool finite(cd a) { return isfinite(a.x) && isfinite(a.y); }

constexpr double kUlp = 2.220446049250313e-16;
constexpr double kSafeMin = 1e-300;

// c real, s complex with  c*x + s*y = r,  -conj(s)*x + c*y = 0.
DENSE_HD inline void givens(cd x, cd y, double& c, cd& s, cd& r) {
  const double ax = cabs(x), ay = cabs(y);
  if (ay == 0.0) { c = 1.0; s = mk(0.0, 0.0); r = x; return; }
  if (ax == 0.0) { c = 0.0; s = scal(conj(y), 1.0 / ay); r = mk(ay, 0.0); return; }
  const double nrm = hypot(ax, ay);
  c = ax / nrm;
  const cd ph = scal(x, 1.0 / ax);            // x/|x|
  s = scal(cmulc(ph, y), 1.0 / nrm);          // (x/|x|) conj(y) / nrm
  r = scal(ph, nrm);
}

// ----------------------------------------------------------------- team types
#ifdef __CUDACC__
struct WarpTeam {
  __device__ int lane() const { return threadIdx.x & 31; }
  static constexpr int size = 32;
  __device__ void sync() const { __syncwarp(); }
};
#endif
struct HostTeam {
  int lane() const { return 0; }
  static constexpr int size = 1;
  void sync() const {}
};

// --------------------------------------------------------- Hessenberg reduction
// A (m x m, ld) <- Z^H A Z upper Hessenberg; Z (m x m, ld) is multiplied from
// the right by the reflectors (pass Z = I to obtain the similarity).
// v: scratch of m entries, sc: scratch of >= 2 doubles.
template <class TM>
DENSE_HD void hessenberg(const TM& tm, cd* A, cd* Z, int m, int ld, cd* v, double* sc) {
  const int lane = tm.lane();
  for (int j = 0; j + 2 < m; ++j) {
    const int L = m - j - 1;   // rows j+1 .. m-1
    if (lane == 0) {
      double nrm2 = 0.0;
      for (int i = 0; i < L; ++i) nrm2 += abs2(A[(j + 1 + i) * ld + j]);
      sc[0] = sqrt(nrm2);
    }
    tm.sync();
    const double alpha = sc[0];
    const cd x0 = A[(j + 1) * ld + j];
    double tail = 0.0;
    tm.sync();
    if (alpha <= kSafeMin) continue;
    const double ax0 = cabs(x0);
    tail = alpha * alpha - ax0 * ax0;
    if (tail <= (kUlp * alpha) * (kUlp * alpha)) continue;  // column already reduced
    const cd ph = ax0 > 0.0 ? scal(x0, 1.0 / ax0) : mk(1.0, 0.0);
    for (int i = lane; i < L; i += tm.size) v[i] = A[(j + 1 + i) * ld + j];
    tm.sync();
    if (lane == 0) v[0] = add(v[0], scal(ph, alpha));
    tm.sync();
    const double tau = 1.0 / (alpha * (alpha + ax0));  // 2 / ||v||^2
    // left: A[j+1:, c] -= tau v (v^H A[j+1:, c]) for c = j..m-1
    for (int c = j + lane; c < m; c += tm.size) {
      cd p = mk(0.0, 0.0);
      for (int i = 0; i < L; ++i) p = add(p, conjmul(v[i], A[(j + 1 + i) * ld + c]));
      p = scal(p, tau);
      for (int i = 0; i < L; ++i) A[(j + 1 + i) * ld + c] = sub(A[(j + 1 + i) * ld + c], mul(v[i], p));
    }
    tm.sync();
    // right: A[r, j+1:] -= tau (A[r, j+1:] v) v^H for all rows; same for Z
    for (int r = lane; r < 2 * m; r += tm.size) {
      cd* M = r < m ? A : Z;
      const int rr = r < m ? r : r - m;
      cd q = mk(0.0, 0.0);
      for (int i = 0; i < L; ++i) q = add(q, mul(M[rr * ld + j + 1 + i], v[i]));
      q = scal(q, tau);
      for (int i = 0; i < L; ++i) M[rr * ld + j + 1 + i] = sub(M[rr * ld + j + 1 + i], cmulc(q, v[i]));
    }
    tm.sync();
    for (int i = 1 + lane; i < L; i += tm.size) A[(j + 1 + i) * ld + j] = mk(0.0, 0.0);
    tm.sync();
  }
}

// ---------------------------------------------------------------- Schur form
// H (m x m upper Hessenberg) -> T upper triangular, Z <- Z Q.  Returns 0 on
// success, -1 if the iteration limit was reached.  sc: >= 8 doubles scratch.
template <class TM>
DENSE_HD int schur_qr(const TM& tm, cd* H, cd* Z, int m, int ld, bool want_z) {
  const int lane = tm.lane();
  int hi = m - 1;
  int iter = 0, total = 0;
  const int max_total = 60 * (m > 1 ? m : 1);
  while (hi > 0) {
    // deflation: largest l <= hi with negligible subdiagonal H[l][l-1]
    int l = hi;
    for (; l > 0; --l) {
      const double sd = cabs(H[l * ld + l - 1]);
      double ref = cabs(H[(l - 1) * ld + l - 1]) + cabs(H[l * ld + l]);
      if (ref == 0.0) ref = 1.0;
      if (sd <= kUlp * ref || sd <= kSafeMin) break;
    }
    tm.sync();
    if (l > 0 && lane == 0) H[l * ld + l - 1] = mk(0.0, 0.0);
    tm.sync();
    if (l == hi) { --hi; iter = 0; continue; }
    if (++total > max_total) return -1;
    ++iter;
    // Wilkinson shift from the trailing 2x2 block of the active window
    const cd a = H[(hi - 1) * ld + hi - 1], b = H[(hi - 1) * ld + hi];
    const cd c = H[hi * ld + hi - 1], d = H[hi * ld + hi];
    cd shift;
    if (iter % 11 == 10) {
      // exceptional shift
      shift = add(d, mk(0.75 * cabs(c), 0.0));
    } else {
      const cd p = scal(sub(a, d), 0.5);
      const cd bc = mul(b, c);
      const cd disc = csqrt(add(mul(p, p), bc));
      const cd den1 = add(p, disc), den2 = sub(p, disc);
      const cd den = cabs(den1) >= cabs(den2) ? den1 : den2;
      shift = cabs(den) > 0.0 ? sub(d, cdiv(bc, den)) : d;
    }
    // implicit single-shift QR sweep on rows/cols l..hi (bulge chase)
    cd x = sub(H[l * ld + l], shift), y = H[(l + 1) * ld + l];
    for (int k = l; k < hi; ++k) {
      if (k > l) { x = H[k * ld + k - 1]; y = H[(k + 1) * ld + k - 1]; }
      double cs; cd sn, rr;
      givens(x, y, cs, sn, rr);
      tm.sync();
      // rows k, k+1 of H, columns from max(l, k-1) to m-1 (full Schur form)
      const int c0 = k > l ? k - 1 : l;
      for (int col = c0 + lane; col < m; col += tm.size) {
        const cd u = H[k * ld + col], w = H[(k + 1) * ld + col];
        H[k * ld + col] = add(scal(u, cs), mul(sn, w));
        H[(k + 1) * ld + col] = sub(scal(w, cs), conjmul(sn, u));
      }
      tm.sync();
      // columns k, k+1 of H for rows 0 .. min(k+2, hi), and of Z for all rows
      const int r1 = (k + 2 < hi ? k + 2 : hi) + 1;
      const int nz = want_z ? m : 0;
      for (int r = lane; r < r1 + nz; r += tm.size) {
        cd* M = r < r1 ? H : Z;
        const int rr = r < r1 ? r : r - r1;
        const cd u = M[rr * ld + k], w = M[rr * ld + k + 1];
        M[rr * ld + k] = add(scal(u, cs), cmulc(w, sn));
        M[rr * ld + k + 1] = sub(scal(w, cs), mul(u, sn));
      }
      tm.sync();
    }
    // uniform decision: every lane scans the whole diagonal
    bool bad = false;
    for (int r = 0; r < m; ++r) bad = bad || !finite(H[r * ld + r]);
    tm.sync();
    if (bad) return -2;
  }
  return 0;
}

// Eigenvectors of upper-triangular T for the eigenvalues T[idx[q]][idx[q]],
// q < cnt: Y[:, q] (ld_y columns) with Y[i][q] = 0 for i > idx[q], Y[idx[q]][q] = 1.
template <class TM>
DENSE_HD void tri_eigvecs(const TM& tm, const cd* T, int m, int ld, const int* idx, int cnt, cd* Y, int ldy) {
  double tn = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j) tn = fmax(tn, cabs(T[i * ld + j]));
  const double small = fmax(kUlp * tn, kSafeMin);
  for (int q = tm.lane(); q < cnt; q += tm.size) {
    const int i0 = idx[q];
    const cd lam = T[i0 * ld + i0];
    for (int i = 0; i < m; ++i) Y[i * ldy + q] = mk(i == i0 ? 1.0 : 0.0, 0.0);
    for (int j = i0 - 1; j >= 0; --j) {
      cd s = mk(0.0, 0.0);
      for (int l = j + 1; l <= i0; ++l) s = add(s, mul(T[j * ld + l], Y[l * ldy + q]));
      cd den = sub(T[j * ld + j], lam);
      if (cabs(den) < small) den = mk(small, 0.0);
      Y[j * ldy + q] = scal(cdiv(s, den), -1.0);
    }
  }
  tm.sync();
}

// Leja ordering (Alg. 2).  Single lane.  theta in/out (d entries), work: d ints.
DENSE_HD inline bool leja_better(cd a, cd b, int ia, int ib, double sa, double sb) {
  if (sa != sb) return sa > sb;
  if (a.x != b.x) return a.x > b.x;
  if (a.y != b.y) return a.y > b.y;
  return ia < ib;
}

DENSE_HD inline void leja_order(cd* theta, int d, int* used, cd* out) {
  for (int i = 0; i < d; ++i) used[i] = 0;
  for (int step = 0; step < d; ++step) {
    int best = -1;
    double bs = 0.0;
    for (int i = 0; i < d; ++i) {
      if (used[i]) continue;
      double sc;
      if (step == 0) {
        sc = cabs(theta[i]);
      } else {
        sc = 0.0;
        for (int j = 0; j < step; ++j) {
          const double dist = cabs(sub(theta[i], out[j]));
          if (dist == 0.0) { sc = -INFINITY; break; }
          sc += log(dist);
        }
      }
      if (best < 0 || leja_better(theta[i], theta[best], i, best, sc, bs)) { best = i; bs = sc; }
    }
    used[best] = 1;
    out[step] = theta[best];
  }
  for (int i = 0; i < d; ++i) theta[i] = out[i];
}

// --------------------------------------------------------- harmonic Ritz problem
// Given the Givens QR of the (k+j+1) x (k+j) matrix G = [[I_k, B], [0, Hbar_j]]
// (rotations cs/sn act on rows k+i, k+i+1; R_H = rotated Hbar, j x j upper
// triangular) and S = What^H Vhat = [[S_top, 0], [S_bot, I_(j+1) x j]], form
// M = R_G^{-1} (Q_G^H S)[0:k+j, :], whose eigenvalues nu are 1/theta for the
// harmonic Ritz values theta (G^H G z = theta G^H S z).
//   Rh: ld_r, element (row i, col c) = Rh[c*ld_r + i]  (column-major, as built per Arnoldi step)
//   B : element (i, c) = B[c*ld_b + i]  (column-major with the solver's leading dimension)
//   Stop: k x k row-major;  Sbot: (j+1) x k row-major
// Output M (row-major, ld) of size (k+j) x (k+j).
template <class TM>
DENSE_HD int harmonic_matrix(const TM& tm, int k, int j, const double* cs, const cd* sn, const cd* Rh, int ld_r,
                             const cd* B, int ld_b, const cd* Stop, const cd* Sbot, cd* M, int ld) {
  const int n = k + j;
  const int lane = tm.lane();
  // X = Q^H S, rows 0..n (one extra row kept during the rotation), stored in M's space + scratch row
  // fill rows 0..n of S into M (row n lives at M[n*ld], the caller provides ld >= n+1 rows)
  for (int e = lane; e < (n + 1) * n; e += tm.size) {
    const int r = e / n, c = e % n;
    cd v = mk(0.0, 0.0);
    if (r < k) {
      if (c < k) v = Stop[r * k + c];
    } else {
      const int rb = r - k;            // row of the lower part, 0..j
      if (c < k) v = Sbot[rb * k + c];
      else if (rb == c - k) v = mk(1.0, 0.0);
    }
    M[r * ld + c] = v;
  }
  tm.sync();
  for (int i = 0; i < j; ++i) {
    const int r0 = k + i, r1 = k + i + 1;
    for (int c = lane; c < n; c += tm.size) {
      const cd u = M[r0 * ld + c], w = M[r1 * ld + c];
      M[r0 * ld + c] = add(scal(u, cs[i]), mul(sn[i], w));
      M[r1 * ld + c] = sub(scal(w, cs[i]), conjmul(sn[i], u));
    }
    tm.sync();
  }
  // back substitution R_G Y = X (rows 0..n-1), R_G = [[I, B], [0, R_H]]; columns in parallel.
  // The pivot test is made by every lane on the same data (uniform return).
  for (int i = 0; i < j; ++i)
    if (!(cabs(Rh[i * ld_r + i]) > kSafeMin)) return -1;
  for (int c = lane; c < n; c += tm.size) {
    for (int i = j - 1; i >= 0; --i) {
      cd s = M[(k + i) * ld + c];
      for (int l = i + 1; l < j; ++l) s = sub(s, mul(Rh[l * ld_r + i], M[(k + l) * ld + c]));
      M[(k + i) * ld + c] = cdiv(s, Rh[i * ld_r + i]);
    }
    for (int i = 0; i < k; ++i) {
      cd s = M[i * ld + c];
      for (int l = 0; l < j; ++l) s = sub(s, mul(B[l * ld_b + i], M[(k + l) * ld + c]));
      M[i * ld + c] = s;
    }
  }
  tm.sync();
  return 0;
}

}  // namespace dense
}  // namespace coarse
