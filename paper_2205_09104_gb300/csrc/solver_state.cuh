// Device-resident state of one Arnoldi cycle and the small dense arrays of
// the solver (shared by dense.cu and solver.cu).
#pragma once

#include "common.cuh"

namespace coarse {

constexpr int kMaxDense = 64;                 // largest restart length m (and k + j)
constexpr int kMaxK = 32;                     // largest recycle dimension k
constexpr int kMaxPoly = 32;                  // largest polynomial degree d
constexpr int kPolyScale = 3 * kMaxDense;     // slot of 1/theta_1 in the chain table

// status bits of a cycle
enum : int { ST_LUCKY = 1, ST_NONFINITE = 2, ST_ZERO = 4, ST_BREAKDOWN = 8 };

struct CycleState {
  int j;        // Arnoldi steps done in this cycle
  int k;        // recycle vectors active in this cycle
  int steps;    // steps allowed
  int stop;     // per-step kernels return at once when set
  int status;   // ST_* bits
  int rstatus;  // result of k_recycle / k_poly_roots (0 = ok)
  int d;        // polynomial degree found by k_poly_roots
  int p1_skip;  // pipelined step: 1 when this step's vector recurrences must not run
  double beta;    // ||r|| at the start of the cycle
  double target;  // least-squares residual that ends the cycle
  double resid;   // current least-squares residual |g_{j+1}|
  double inv_h;   // 1 / h_{j+1,j} (1 / beta before the first step)
  double wnorm2;  // ||w||^2 after the second Gram-Schmidt pass
  double spare[3];
};

// Small dense arrays, all FP64 complex unless stated.  Column-major for the
// matrices built one Arnoldi column at a time.
struct Dense {
  double2* H;      // Hbar, (ldh) x m, H[col*ldh + row]
  double2* R;      // Givens-rotated Hbar (upper triangular)
  double* cs;      // rotation cosines, m
  double2* sn;     // rotation sines, m
  double2* g;      // rotated right-hand side beta e1, m+1
  double2* B;      // B_k = C^H A V, B[col*ldb + row]
  double2* ycoef;  // [y_U (k); y_V (j)]
  double2* z;      // Hbar y_V, j+1
  double2* coefC;  // (k+j+1) x knew
  double2* coefU;  // (k+j) x knew
  double2* theta;  // Leja-ordered harmonic Ritz values
  double2* polyc;  // chain coefficients, 3 per step + scale slot
  int ldh;
  int ldb;
};

int launch_cycle_init(CycleState* st, int k, int steps, const double* rnorm2, double target, double2* g,
                      cudaStream_t s);
int launch_step_finalize(CycleState* st, const double2* h1, const double2* h2, const Dense& d, cudaStream_t s);
// Latency-1 pipelined Arnoldi (Sec. 3.5): from the fused reduction of step i (h = [C, V]^H v^a_{i-1}
// and ||v^a_{i-1}||^2) form t = ||v^a||^2 - sum |h|^2 into st->wnorm2 for the finalize; t below
// minus its rounding (tol_u: unit roundoff of the vectors) is a breakdown that stops the cycle.
int launch_p1_prep(CycleState* st, const double2* h, const double* nva, double tol_u, cudaStream_t s);
int launch_cycle_solve(const CycleState* st, const Dense& d, cudaStream_t s);
int launch_recycle(CycleState* st, const Dense& d, const double2* SW, int ldsw, int knew, cudaStream_t s);
int launch_poly_roots(CycleState* st, const Dense& d, int dmax, cudaStream_t s);
int launch_axpy(int prec64, const void* x, void* y, double2 alpha, int N, const int* stop, cudaStream_t s);

}  // namespace coarse
