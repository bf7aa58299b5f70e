// Odd-even reduced system with block-Jacobi left preconditioning (Sec. 2, Sec. 3.2): arguments
// of the fused half apply and the launchers (oddeven.cu).
#pragma once

#include "common.cuh"

namespace coarse {

struct EoArgs {
  const void* blocks;   // [V][5][n][n] of the block type
  const void* inv;      // [V][n][n] inverses of the diagonal blocks A_x + i mu sigma3, same type
  const int4* rec;      // [V][4] neighbour records (coarse_op::eo_rec): even list, then odd list
  int* err;             // raised (1) if a bounded wait of the prefetching variant ran out
  int V;
  int out_par;          // parity of the output sites (0 even, 1 odd)
  const void* v;        // hop input, compressed on the other parity (nullptr: no hops)
  const void* z;        // optional: the inverse acts on z - h instead of h
  const void* base;     // optional: y = base - u instead of y = u
  void* y;              // output, compressed on out_par
  int mode;             // ApplyMode epilogue on y (chain input x = base)
  void* acc;
  const double2* coef;
  const int* stop;      // optional device flag: return if set
};

// Index of the inverse set for the twisted mass mu_eff: 0 for +mu (and for mu = 0), 1 for -mu.
inline int eo_sign(const coarse_op* op, double mu_eff) { return (op->mu != 0.0 && mu_eff != op->mu) ? 1 : 0; }
// Inverses of the diagonal blocks for the twisted mass mu_eff, in every enabled precision
// (synchronises s the first time for each mass sign).
int eo_prepare(coarse_op* op, double mu_eff, cudaStream_t s);
int launch_eo_half(int prec, int n, const EoArgs& a, cudaStream_t s);
int launch_eo_split(int v64, const void* full, const int* sites, int V, int n, void* ev, void* od, cudaStream_t s);
int launch_eo_merge(int v64, const void* ev, const void* od, const int* sites, int V, int n, void* full, cudaStream_t s);
// y = S x (compressed even vectors; t: odd scratch), with the polynomial-chain epilogue
int launch_eo_schur(const coarse_op* op, int prec, double mu_eff, const void* x, void* y, void* t, int mode, void* acc,
                    const double2* coef, const int* stop, cudaStream_t s);

}  // namespace coarse
