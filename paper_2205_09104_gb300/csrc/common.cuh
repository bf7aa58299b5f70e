// Internal declarations shared by the translation units of the coarse library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/coarse.h"

namespace coarse {

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ float2 cmk(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
template <class C> __host__ __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class C> __host__ __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <class C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// conj(a) * b
template <class C> __host__ __device__ __forceinline__ C cconjmul(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <class C> __host__ __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
template <class C, class S> __host__ __device__ __forceinline__ C cscale(C a, S s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <class C> __host__ __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

// acc += a * b  (complex multiply-accumulate, 4 FMAs)
template <class C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class C> __host__ __device__ __forceinline__ void cfma_conj(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// BF16 complex storage element: (re, im) as two bf16 in 4 bytes
struct __align__(4) cbf16 { __nv_bfloat16 x, y; };

// ------------------------------------------------------------------ error state
void set_error(const char* fmt, ...);
void note_launch();          // counts kernels launched by the library
void note_launches(long long n);  // ... n at once (kernels of a replayed CUDA graph)
int sm_count();              // multiprocessors of the current device (cached)
long long launches_so_far();
int cuda_fail(cudaError_t e, const char* what);
#define COARSE_CUDA(call)                                      \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return ::coarse::cuda_fail(_e, #call); \
  } while (0)

// ---------------------------------------------------------------- precision data
// Block storage of one precision: [V][5][n][n], block 0 = self, 1..4 = forward hops.
struct Blocks {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Solver;  // per-precision solver state, defined in solver.cu

}  // namespace coarse

struct coarse_op {
  int dims[4];
  int V;
  int nv;
  int n;
  double mu;
  int max_nrhs;
  uint32_t precisions;
  int* nb = nullptr;                // device int32 [V][8]
  coarse::Blocks blk[3];            // FP64, FP32, BF16 copies
  coarse::Blocks mrhs;              // BF16 blocks in the tensor-core fragment layout (BF16 and max_nrhs > 1)
  coarse::Blocks mrhs_x;            // packed BF16 columns of one multi-RHS pass (scratch of the multi-RHS apply)
  coarse::Blocks umma;              // BF16 blocks as tcgen05 core-matrix planes (n = 32, 48; BF16 and max_nrhs > 1)
  // odd-even reduction (all extents even): site lists and inverses of the diagonal blocks
  int* eo_sites = nullptr;          // device [V]: even sites, then odd sites, each in increasing order
  int* eo_half = nullptr;           // device [V]: position of each site in its parity's list
  int4* eo_rec = nullptr;           // device [V][4]: for the q-th site x of the (even, odd) list and
                                    // direction mu, {half index of x+mu, x-mu, half index of x-mu, x}
  coarse::Blocks inv[2][3];         // [mass sign: +mu, -mu][precision]: [V][n][n] inverses of A_x +- i mu sigma3
  int inv_ok[2] = {0, 0};           // inverses of that sign valid for the current blocks
  void* eo_scratch = nullptr;       // FP32 work vectors of odd-even solves (3 N complex64)
  coarse::Solver* eo_solver[3] = {nullptr, nullptr, nullptr};
  coarse::Solver* eo_adj_solver[3] = {nullptr, nullptr, nullptr};  // sigma3 D_c(-mu) sigma3 for mu != 0
  coarse::Solver* solver[3] = {nullptr, nullptr, nullptr};
  coarse::Solver* adj_solver[3] = {nullptr, nullptr, nullptr};  // sigma3 D_c(-mu) sigma3 for mu != 0
  double2* work64 = nullptr;        // 3 FP64 work vectors of V*n: residual, generator scratch, sigma3 temp
  double* red = nullptr;            // FP64 reduction partials
  double* norms = nullptr;          // device norms (||r||^2, ||b||^2, gamma5 defect, ...)
  double2* coef = nullptr;          // device constants: {-1, 1} for r = b - D x
  unsigned* counter = nullptr;      // last-block counter of the op-level reductions
  void* apply_scratch = nullptr;    // 5 * V * n complex128: pull partials and pushes of the stencil
  int* apply_cnt = nullptr;         // V arrival counters of the stencil (zero between launches), then an error flag
  int device = 0;
};

namespace coarse {

// ----------------------------------------------------------------- apply kernels
// Epilogue of the stencil apply.
enum ApplyMode : int {
  APPLY_PLAIN = 0,   // y = D x
  APPLY_AXPBY = 1,   // y = alpha * D x + beta * z   (alpha, beta complex, from coef[0], coef[1])
  APPLY_POLY = 2,    // chain step: y = x - c0 * D x ;  acc = acc + c1 * y  (c0, c1 from coef)
  APPLY_POLY_FIRST = 3  // first chain step: y = x - c0 * D x ; acc = c2 * x + c1 * y
};

struct ApplyArgs {
  const void* blocks;   // [V][5][n][n] of the block type
  const int* nb;        // [V][8]
  const void* x;        // vector in
  void* y;              // vector out
  const void* z;        // AXPBY addend
  void* acc;            // POLY accumulator (in/out)
  const double2* coef;  // device coefficients
  double mu;            // twisted mass (sign already applied)
  int V;
  int mode;
  int adjoint;          // 1: y = sigma3 D(-mu) sigma3 x  (mu sign handled by caller), i.e. D^H
  const int* stop;      // optional device flag: return immediately if *stop != 0
  void* part;           // scratch [V][n] pull partials (vector-accumulator type)
  void* push;           // scratch [4][V][n] pushes to the forward neighbours
  int* cnt;             // [V] arrival counters, zero between launches
  int* err;             // raised (1) if a bounded wait of the TMA-staged kernel expired
};

int launch_apply(int prec, int n, const ApplyArgs& a, cudaStream_t s);

// Arguments of a plain y = D x launch on operator `op` with the blocks of precision `prec`.
inline ApplyArgs make_apply_args(const coarse_op* op, int prec, const void* x, void* y) {
  ApplyArgs a;
  a.blocks = op->blk[prec].ptr;
  a.nb = op->nb;
  a.x = x;
  a.y = y;
  a.z = nullptr;
  a.acc = nullptr;
  a.coef = nullptr;
  a.mu = op->mu;
  a.V = op->V;
  a.mode = APPLY_PLAIN;
  a.adjoint = 0;
  a.stop = nullptr;
  a.part = op->apply_scratch;
  a.push = (char*)op->apply_scratch + (size_t)op->V * op->n * (prec == COARSE_PREC_FP64 ? 16 : 8);
  a.cnt = op->apply_cnt;
  a.err = op->apply_cnt + op->V;
  return a;
}
int launch_apply_mrhs_bf16(const coarse_op* op, const void* x, void* y, int nrhs, int adjoint, cudaStream_t s);
int launch_pack_mrhs(const coarse_op* op, cudaStream_t s);  // refresh op->mrhs from the BF16 blocks
// Reads and clears the operator's stencil error flag (synchronises s); COARSE_ERR_TIMEOUT if raised.
int take_stencil_flag(const coarse_op* op, cudaStream_t s);

// ------------------------------------------------------------------ BLAS kernels
// Vectors of the solver: complex64 (float2) or complex128 (double2), length N.
template <class C> struct VecList { const C* const* v; int count; };

int launch_multidot(int prec64, const void* const* q, int nq, const void* w, int N, double2* out,
                    double* wnorm2, double* partial, unsigned* counter, const int* stop, cudaStream_t s);
// w -= (negate) / += sum_i q_i h_i; mode 0: nothing else, 1: ||w||^2 -> wnorm2, 2: out = Q^H w and
// ||w||^2 of the updated w (fused second Gram-Schmidt pass).
int launch_update(int prec64, const void* const* q, int nq, const double2* h, int negate, void* w, int N,
                  int mode, double2* out_dots, double* wnorm2, double* partial, unsigned* counter,
                  const int* stop, cudaStream_t s);
int max_reduction_chunks(int N);  // partial-array columns the reductions use for length N
int launch_combine(int prec64, const void* const* in, int nin, const double2* coef, int ldc, void* const* out,
                   int nout, int accumulate, int N, const int* stop, cudaStream_t s);
int launch_scale(int prec64, const void* x, const double* inv_or_null, double2 alpha, void* y, int N,
                 const int* gate, int gate_val, cudaStream_t s);
int launch_norm2(int prec64, const void* x, int N, double* out, double* partial, unsigned* counter,
                 cudaStream_t s);
int launch_to_low(const double2* x64, const double* norm_dev, float2* y32, int N, cudaStream_t s);
int launch_add_low(double2* x64, const double* norm_dev, const float2* e32, int N, cudaStream_t s);
int launch_sigma3(int prec64, const void* x, void* y, int n, int V, cudaStream_t s);
int launch_fill_gaussian(double2* x, int N, uint64_t seed, cudaStream_t s);
int launch_copy_to(int prec64, const double2* x64, void* y, int N, cudaStream_t s);
int launch_check_finite(int prec64, const void* x, int N, int* flag, cudaStream_t s);

// ------------------------------------------------------------------ conversions
int launch_ingest(const double2* self_b, const double2* hop_b, int gamma5_only, int V, int n, const int* nb,
                  void* out64, void* out32, void* out16, cudaStream_t s);
int launch_gamma5_defect(const double2* self_b, const double2* hop_b, int V, int n, const int* nb,
                         double* out2, cudaStream_t s);
int launch_block_grad(const double2* lam, const double2* x, const int* nb, int V, int n, int nhop, double2* g_self,
                      double2* g_hop, cudaStream_t s);

}  // namespace coarse
