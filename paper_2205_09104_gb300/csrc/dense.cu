// Device kernels for the small dense FP64 work of the Krylov solver; all of
// them run on one CTA and keep their matrices in shared or global memory.
//   k_cycle_init      start of an Arnoldi cycle: beta = ||r||, g = beta e1
//   k_step_finalize   Arnoldi column j: H and B entries from the two CGS passes,
//                     h_{j+1,j} = ||w||, Givens update of the least-squares
//                     problem (Sec. 3.1), residual estimate, stop flag
//   k_cycle_solve     y = R^{-1} g, y_U = -B y_V (paper form G = [[I, B], [0, Hbar]]),
//                     z = Hbar y_V for the residual update (Sec. 3.4, step 4)
//   k_recycle         harmonic Ritz vectors of the cycle and the new U_k, C_k
//                     coefficients (Sec. 3.4, steps 1-2)
//   k_poly_roots      harmonic Ritz values of a d-step Arnoldi, Leja order and the
//                     coefficients of the q(A) chain (Sec. 3.3, Alg. 2, Alg. 3)
#include "common.cuh"
#include "dense.cuh"
#include "solver_state.cuh"
#include "batch.cuh"

namespace coarse {
namespace {

using namespace dense;

__global__ void k_cycle_init(CycleState* st, int k, int steps, const double* rnorm2, double target, double2* g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(fmax(*rnorm2, 0.0));
  st->j = 0;
  st->k = k;
  st->steps = steps;
  st->stop = 0;
  st->status = 0;
  st->beta = beta;
  st->target = target;
  st->resid = beta;
  st->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
  g[0] = make_double2(beta, 0.0);
  if (!(beta > 0.0) || !isfinite(beta)) {
    st->stop = 1;
    st->status = isfinite(beta) ? ST_ZERO : ST_NONFINITE;
  }
}

// One warp.  Loads and stores are lane-parallel; only the j rotations of the new
// column (inherently sequential) and the new rotation run on lane 0.
__device__ void finalize_warp(CycleState* st, const double2* h1, const double2* h2, const Dense& d) {
  __shared__ double2 col[kMaxDense + 2];
  __shared__ double csh[kMaxDense];
  __shared__ double2 snh[kMaxDense];
  __shared__ double hn2s;
  const int lane = threadIdx.x & 31;
  // all scalar state in one round trip, then everything indexed by j in a second one
  const int stop0 = st->stop, j = st->j, k = st->k, steps = st->steps, status0 = st->status;
  const double wn2_raw = st->wnorm2, target = st->target;
  if (stop0) return;  // every lane reads the same flag
  const int ldh = d.ldh;
  const double2 gj = d.g[j];
  double hn2 = 0.0;
  for (int i = lane; i < k; i += 32) {
    const double2 b = h2 ? add(h1[i], h2[i]) : h1[i];
    d.B[j * d.ldb + i] = b;
    hn2 += abs2(b);
  }
  for (int i = lane; i <= j; i += 32) {
    const double2 h = h2 ? add(h1[k + i], h2[k + i]) : h1[k + i];
    d.H[j * ldh + i] = h;
    col[i] = h;
    hn2 += abs2(h);
  }
  for (int i = lane; i < j; i += 32) {
    csh[i] = d.cs[i];
    snh[i] = d.sn[i];
  }
  for (int off = 16; off > 0; off >>= 1) hn2 += __shfl_xor_sync(0xffffffffu, hn2, off);
  __syncwarp();
  if (lane == 0) {
    const double wn2 = fmax(wn2_raw, 0.0);
    const double hj1 = sqrt(wn2);
    hn2 += wn2;
    hn2s = hn2;
    d.H[j * ldh + j + 1] = make_double2(hj1, 0.0);
    col[j + 1] = make_double2(hj1, 0.0);
    for (int i = 0; i < j; ++i) {
      const double2 u = col[i], w = col[i + 1];
      col[i] = add(scal(u, csh[i]), mul(snh[i], w));
      col[i + 1] = sub(scal(w, csh[i]), conjmul(snh[i], u));
    }
    double c;
    double2 sg, r;
    givens(col[j], col[j + 1], c, sg, r);
    d.cs[j] = c;
    d.sn[j] = sg;
    col[j] = r;
    col[j + 1] = make_double2(0.0, 0.0);
    d.g[j] = scal(gj, c);
    d.g[j + 1] = scal(conjmul(sg, gj), -1.0);
    const double resid = cabs(d.g[j + 1]);
    st->resid = resid;
    st->inv_h = hj1 > 0.0 ? 1.0 / hj1 : 0.0;
    int stop = 0, status = status0;
    if (!isfinite(hn2) || !isfinite(resid)) {
      stop = 1;
      status |= ST_NONFINITE;
    } else {
      if (resid <= target) stop = 1;
      if (hj1 <= 1e-14 * sqrt(hn2)) {  // invariant Krylov space: the least-squares solution is exact
        stop = 1;
        status |= ST_LUCKY;
      }
      if (j + 1 >= steps) stop = 1;
    }
    st->status = status;
    st->stop = stop;
  }
  __syncwarp();
  for (int i = lane; i <= j + 1; i += 32) d.R[j * ldh + i] = col[i];
  __syncwarp();
  if (lane == 0) st->j = j + 1;  // last: the normalisation kernel of this step keys on st->j == j + 1
}

__global__ void __launch_bounds__(32) k_step_finalize(CycleState* st, const double2* h1, const double2* h2, Dense d) {
  finalize_warp(st, h1, h2, d);
}

__global__ void __launch_bounds__(32) kb_finalize(const BSolve* S) {
  const BSolve& s = S[blockIdx.x];
  finalize_warp(s.st, s.h1, s.h2, s.dn);
}

// One warp: y = R^{-1} g by column-oriented back substitution (R staged in shared memory,
// lane r owns right-hand-side rows r and r + 32), then y_U = -B y_V and z = Hbar y_V.
__device__ void cycle_solve_warp(const CycleState* st, const Dense& d) {
  extern __shared__ double2 Rs[];  // kMaxDense columns of d.ldh entries
  __shared__ double2 ys[kMaxDense];
  const int lane = threadIdx.x & 31;
  const int j = st->j, k = st->k, ldh = d.ldh;
  for (int e = lane; e < j * ldh; e += 32) Rs[e] = d.R[e];
  double2 x0 = lane < j ? d.g[lane] : make_double2(0.0, 0.0);
  double2 x1 = lane + 32 < j ? d.g[lane + 32] : make_double2(0.0, 0.0);
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    const double2 xi_lo = make_double2(__shfl_sync(0xffffffffu, x0.x, i & 31), __shfl_sync(0xffffffffu, x0.y, i & 31));
    const double2 xi_hi = make_double2(__shfl_sync(0xffffffffu, x1.x, i & 31), __shfl_sync(0xffffffffu, x1.y, i & 31));
    const double2 xi = i < 32 ? xi_lo : xi_hi;
    const double2 piv = Rs[i * ldh + i];
    const double2 yi = cabs(piv) > kSafeMin ? cdiv(xi, piv) : make_double2(0.0, 0.0);
    if (lane == 0) ys[i] = yi;
    if (lane < i) x0 = sub(x0, mul(Rs[i * ldh + lane], yi));
    if (lane + 32 < i) x1 = sub(x1, mul(Rs[i * ldh + lane + 32], yi));
  }
  __syncwarp();
  double2* y = d.ycoef + k;  // y_V
  for (int i = lane; i < j; i += 32) y[i] = ys[i];
  for (int i = lane; i < k; i += 32) {
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < j; ++l) s = add(s, mul(d.B[l * d.ldb + i], ys[l]));
    d.ycoef[i] = scal(s, -1.0);
  }
  for (int i = lane; i <= j; i += 32) {
    double2 s = make_double2(0.0, 0.0);
    for (int l = (i > 0 ? i - 1 : 0); l < j; ++l) s = add(s, mul(d.H[l * ldh + i], ys[l]));
    d.z[i] = s;
  }
}

__global__ void __launch_bounds__(32) k_cycle_solve(const CycleState* st, Dense d) { cycle_solve_warp(st, d); }

__global__ void __launch_bounds__(32) kb_cycle_solve(const BSolve* S) {
  const BSolve& s = S[blockIdx.x];
  if (!bgate(s, BG_TAIL)) return;
  cycle_solve_warp(s.st, s.dn);
}

// start of a cycle for every inner-active solve; inactive solves are stopped.
// target: relative to the inner right-hand side, whose norm is 1 at the start of a refinement
// step (per-solve target in norm2[3]).
__global__ void kb_cycle_init(const BSolve* S, int m) {
  const BSolve& s = S[blockIdx.x];
  if (threadIdx.x != 0) return;
  CycleState* st = s.st;
  st->j = 0;
  st->rstatus = 0;
  if (!s.flags[0]) {
    st->stop = 1;
    st->status = 0;
    return;
  }
  const double beta = sqrt(fmax(s.norm2[0], 0.0));
  st->k = s.kc;
  st->steps = s.kc > 0 ? m - s.kc : m;
  st->stop = 0;
  st->status = 0;
  st->beta = beta;
  st->target = s.norm2[3];
  st->resid = beta;
  st->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
  s.dn.g[0] = make_double2(beta, 0.0);
  if (!(beta > 0.0) || !isfinite(beta)) {
    st->stop = 1;
    st->status = isfinite(beta) ? ST_ZERO : ST_NONFINITE;
  }
}

__global__ void kb_step_inc(int* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

// Harmonic Ritz vectors of the cycle just finished and the coefficients of
// the new recycle space: C_new = What Q2, U_new = Vhat (P R2^{-1}).
// Shared memory: M ((n+1) x LD), Z (n x LD), Y (n x knew), small scratch.
__global__ void __launch_bounds__(32) k_recycle(CycleState* st, Dense d, const double2* SW, int ldsw, int knew) {
  extern __shared__ double2 sm[];
  constexpr int LD = kMaxDense;
  const int k = st->k, j = st->j, n = k + j;
  double2* M = sm;                       // (LD+1) x LD
  double2* Z = M + (LD + 1) * LD;        // LD x LD
  double2* Y = Z + LD * LD;              // LD x kMaxK
  double2* Stop = Y + LD * kMaxK;        // k x k
  double2* Sbot = Stop + kMaxK * kMaxK;  // (j+1) x k
  double2* v = Sbot + (LD + 1) * kMaxK;  // LD
  double* sc = reinterpret_cast<double*>(v + LD + 1);
  int* idx = reinterpret_cast<int*>(sc + 8);
  WarpTeam tm;
  const int lane = tm.lane();
  if (n < knew || knew <= 0 || n > LD) {
    if (lane == 0) st->rstatus = 1;
    return;
  }
  for (int e = lane; e < k * k; e += 32) {
    const int r = e / k, c = e % k;
    Stop[r * k + c] = SW[c * ldsw + r];
  }
  for (int e = lane; e < (j + 1) * k; e += 32) {
    const int r = e / k, c = e % k;
    Sbot[r * k + c] = SW[c * ldsw + k + r];
  }
  tm.sync();
  int rc = harmonic_matrix(tm, k, j, d.cs, d.sn, d.R, d.ldh, d.B, d.ldb, Stop, Sbot, M, LD);
  if (rc) {
    if (lane == 0) st->rstatus = 2;
    return;
  }
  for (int e = lane; e < n * LD; e += 32) Z[e] = make_double2((e / LD) == (e % LD) ? 1.0 : 0.0, 0.0);
  tm.sync();
  hessenberg(tm, M, Z, n, LD, v, sc);
  rc = schur_qr(tm, M, Z, n, LD, true);
  if (rc) {
    if (lane == 0) st->rstatus = 3;
    return;
  }
  // the knew eigenvalues nu of largest modulus (theta = 1/nu of smallest modulus)
  if (lane == 0) {
    for (int q = 0; q < knew; ++q) {
      int best = -1;
      double bm = -1.0;
      for (int i = 0; i < n; ++i) {
        bool used = false;
        for (int p = 0; p < q; ++p) used = used || (idx[p] == i);
        const double a = cabs(M[i * LD + i]);
        if (!used && a > bm) { bm = a; best = i; }
      }
      idx[q] = best;
    }
  }
  tm.sync();
  tri_eigvecs(tm, M, n, LD, idx, knew, Y, kMaxK);
  // P = Z Y  (n x knew) into M's space (T is no longer read), then unit columns
  double2* P = M;
  for (int e = lane; e < n * knew; e += 32) {
    const int r = e / knew, q = e % knew;
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < n; ++l) s = add(s, mul(Z[r * LD + l], Y[l * kMaxK + q]));
    P[e] = s;
  }
  tm.sync();
  for (int q = lane; q < knew; q += 32) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += abs2(P[r * knew + q]);
    s = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int r = 0; r < n; ++r) P[r * knew + q] = scal(P[r * knew + q], s);
  }
  tm.sync();
  // GP = G P, G = [[I_k, B], [0, Hbar]]  ((n+1) x knew), into Z's space
  double2* GP = Z;
  for (int e = lane; e < (n + 1) * knew; e += 32) {
    const int r = e / knew, q = e % knew;
    double2 s = make_double2(0.0, 0.0);
    if (r < k) {
      s = P[r * knew + q];
      for (int l = 0; l < j; ++l) s = add(s, mul(d.B[l * d.ldb + r], P[(k + l) * knew + q]));
    } else {
      const int rr = r - k;
      for (int l = (rr > 0 ? rr - 1 : 0); l < j; ++l) s = add(s, mul(d.H[l * d.ldh + rr], P[(k + l) * knew + q]));
    }
    GP[r * knew + q] = s;
  }
  tm.sync();
  // modified Gram-Schmidt QR of GP: Q2 in place, R2 (knew x knew) in Y
  double2* R2 = Y;
  for (int q = 0; q < knew; ++q) {
    for (int p = 0; p < q; ++p) {
      if (lane == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int r = 0; r <= n; ++r) s = add(s, conjmul(GP[r * knew + p], GP[r * knew + q]));
        R2[p * knew + q] = s;
      }
      tm.sync();
      const double2 s = R2[p * knew + q];
      for (int r = lane; r <= n; r += 32) GP[r * knew + q] = sub(GP[r * knew + q], mul(GP[r * knew + p], s));
      tm.sync();
    }
    if (lane == 0) {
      double s = 0.0;
      for (int r = 0; r <= n; ++r) s += abs2(GP[r * knew + q]);
      sc[0] = sqrt(s);
      R2[q * knew + q] = make_double2(sc[0], 0.0);
      for (int p = q + 1; p < knew; ++p) R2[p * knew + q] = make_double2(0.0, 0.0);
    }
    tm.sync();
    const double nr = sc[0];
    tm.sync();
    if (!(nr > 1e-13)) {
      if (lane == 0) st->rstatus = 4;
      return;
    }
    for (int r = lane; r <= n; r += 32) GP[r * knew + q] = scal(GP[r * knew + q], 1.0 / nr);
    tm.sync();
  }
  // outputs: coefC = Q2 ((n+1) x knew), coefU = P R2^{-1} (n x knew)
  for (int e = lane; e < (n + 1) * knew; e += 32) d.coefC[e] = GP[e];
  for (int r = lane; r < n; r += 32) {
    for (int q = 0; q < knew; ++q) {
      double2 s = P[r * knew + q];
      for (int p = 0; p < q; ++p) s = sub(s, mul(d.coefU[r * knew + p], R2[p * knew + q]));
      d.coefU[r * knew + q] = cdiv(s, R2[q * knew + q]);
    }
  }
  if (lane == 0) st->rstatus = 0;
}

__global__ void __launch_bounds__(32) k_poly_roots(CycleState* st, Dense d, int dmax) {
  extern __shared__ double2 sm[];
  constexpr int LD = kMaxDense;
  double2* M = sm;                 // (LD+1) x LD
  double2* v = M + (LD + 1) * LD;  // LD
  double2* out = v + LD;           // LD
  double* sc = reinterpret_cast<double*>(out + LD);
  int* used = reinterpret_cast<int*>(sc + 8);
  WarpTeam tm;
  const int lane = tm.lane();
  const int j = st->j;
  if (j <= 0 || j > dmax) {
    if (lane == 0) { st->rstatus = 1; st->d = 0; }
    return;
  }
  int rc = harmonic_matrix(tm, 0, j, d.cs, d.sn, d.R, d.ldh, d.B, d.ldb, nullptr, nullptr, M, LD);
  if (rc) {
    if (lane == 0) { st->rstatus = 2; st->d = 0; }
    return;
  }
  hessenberg(tm, M, nullptr, j, LD, v, sc);
  rc = schur_qr(tm, M, nullptr, j, LD, false);
  if (rc) {
    if (lane == 0) { st->rstatus = 3; st->d = 0; }
    return;
  }
  if (lane == 0) {
    for (int i = 0; i < j; ++i) {
      const double2 nu = M[i * LD + i];
      v[i] = cabs(nu) > kSafeMin ? cdiv(make_double2(1.0, 0.0), nu) : make_double2(1e300, 0.0);
    }
    leja_order(v, j, used, out);
    for (int i = 0; i < j; ++i) d.theta[i] = v[i];
    // chain step i (1-based, i < j): c0 = 1/theta_i, c1 = 1/theta_{i+1}, c2 = 1/theta_1
    const double2 one = make_double2(1.0, 0.0);
    for (int i = 1; i < j; ++i) {
      d.polyc[3 * (i - 1) + 0] = cdiv(one, v[i - 1]);
      d.polyc[3 * (i - 1) + 1] = cdiv(one, v[i]);
      d.polyc[3 * (i - 1) + 2] = cdiv(one, v[0]);
    }
    d.polyc[kPolyScale] = cdiv(one, v[0]);  // degree one: q = 1/theta_1
    st->d = j;
    st->rstatus = 0;
  }
}

}  // namespace

int launch_cycle_init(CycleState* st, int k, int steps, const double* rnorm2, double target, double2* g,
                      cudaStream_t s) {
  k_cycle_init<<<1, 32, 0, s>>>(st, k, steps, rnorm2, target, g);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

// Sec. 3.5: t = ||v^a_{i-1}||^2 - sum_j |b_j|^2 - sum_j |h_j|^2 with the coefficients of the fused
// reduction; t < -round (round = 8 (i + k + 1) u ||v^a||^2) is a breakdown: the cycle stops with the
// steps before this one; |t| <= round counts as an invariant subspace (h_{i,i-1} = 0).
__global__ void __launch_bounds__(32) k_p1_prep(CycleState* st, const double2* h, const double* nva, double tol_u) {
  const int lane = threadIdx.x & 31;
  const int stop = st->stop, j = st->j, k = st->k;
  if (stop) {
    if (lane == 0) st->p1_skip = 1;
    return;
  }
  double s2 = 0.0;
  for (int i = lane; i < k + j + 1; i += 32) s2 += abs2(h[i]);
  for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  if (lane != 0) return;
  const double n2 = *nva;
  const double t = n2 - s2;
  const double round = 8.0 * (double)(j + k + 2) * tol_u * n2;
  if (!isfinite(t)) {
    st->stop = 1;
    st->status |= ST_NONFINITE;
    st->p1_skip = 1;
  } else if (t < -round) {
    st->stop = 1;
    st->status |= ST_BREAKDOWN;
    st->p1_skip = 1;
  } else {
    st->wnorm2 = t > round ? t : 0.0;
    st->p1_skip = 0;
  }
}

int launch_p1_prep(CycleState* st, const double2* h, const double* nva, double tol_u, cudaStream_t s) {
  k_p1_prep<<<1, 32, 0, s>>>(st, h, nva, tol_u);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_step_finalize(CycleState* st, const double2* h1, const double2* h2, const Dense& d, cudaStream_t s) {
  k_step_finalize<<<1, 32, 0, s>>>(st, h1, h2, d);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_cycle_solve(const CycleState* st, const Dense& d, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = sizeof(double2) * (size_t)kMaxDense * d.ldh;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_cycle_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_cycle_solve<<<1, 32, smem, s>>>(st, d);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

size_t recycle_smem() {
  constexpr int LD = kMaxDense;
  return sizeof(double2) * ((size_t)(LD + 1) * LD + (size_t)LD * LD + (size_t)LD * kMaxK + (size_t)kMaxK * kMaxK +
                            (size_t)(LD + 1) * kMaxK + LD + 1) +
         8 * sizeof(double) + kMaxK * sizeof(int) + 64;
}

size_t poly_smem() {
  constexpr int LD = kMaxDense;
  return sizeof(double2) * ((size_t)(LD + 1) * LD + 2 * LD) + 8 * sizeof(double) + LD * sizeof(int) + 64;
}

int launch_recycle(CycleState* st, const Dense& d, const double2* SW, int ldsw, int knew, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = recycle_smem();
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_recycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_recycle<<<1, 32, smem, s>>>(st, d, SW, ldsw, knew);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_poly_roots(CycleState* st, const Dense& d, int dmax, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = poly_smem();
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_poly_roots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_poly_roots<<<1, 32, smem, s>>>(st, d, dmax);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace coarse

namespace coarse {

int launch_bcycle_init(const BSolve* S, int nsolves, int m, double /*target*/, cudaStream_t s) {
  if (nsolves <= 0) return COARSE_OK;
  kb_cycle_init<<<nsolves, 32, 0, s>>>(S, m);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_bfinalize(const BSolve* S, int nsolves, cudaStream_t s) {
  if (nsolves <= 0) return COARSE_OK;
  kb_finalize<<<nsolves, 32, 0, s>>>(S);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_bcycle_solve(const BSolve* S, int nsolves, cudaStream_t s) {
  if (nsolves <= 0) return COARSE_OK;
  static bool attr = false;
  const size_t smem = sizeof(double2) * (size_t)kMaxDense * (kMaxDense + 1);
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(kb_cycle_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  kb_cycle_solve<<<nsolves, 32, smem, s>>>(S);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_step_inc(int* step, cudaStream_t s) {
  kb_step_inc<<<1, 32, 0, s>>>(step);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace coarse
