/*
 * coarse.h -- C ABI of the GB300 coarsest-level solver for aggregation-based
 * multigrid (coarse Wilson-clover / twisted-mass Dirac stencil D_c).
 *
 * Paper: "Coarsest-level improvements in multigrid for lattice QCD on
 * large-scale computers", arXiv:2205.09104.
 *
 * General conventions
 *   - Every pointer named as "device" must point to memory of the current CUDA
 *     device; every "host" pointer to host memory.  Streams are cudaStream_t
 *     passed as void* (NULL = legacy default stream).
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = 2 x double,
 *     complex64 = 2 x float.
 *   - Lattice: dims[4] = (L0, L1, L2, L3), V = L0 L1 L2 L3 sites, site index
 *     x = x0 + L0*(x1 + L1*(x2 + L2*x3)), periodic boundaries.
 *   - n = 2*nv unknowns per site: the nv chirality-+ dofs first, then nv
 *     chirality-- dofs; sigma3 = diag(+1 x nv, -1 x nv).
 *   - Vectors are [nrhs][V][n] complex, contiguous.
 *   - Return value: COARSE_OK (0) or a negative coarse_status.  No call aborts
 *     or throws; the message of the last failure on the calling thread is
 *     returned by coarse_last_error().
 */
#ifndef COARSE_H
#define COARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct coarse_op coarse_op; /* opaque operator handle */

typedef enum {
  COARSE_OK = 0,
  COARSE_ERR_INVALID_ARG = -1,   /* bad pointer, size or parameter */
  COARSE_ERR_OOM = -2,           /* device allocation failed */
  COARSE_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  COARSE_ERR_NOT_CONVERGED = -4, /* tolerance not reached; x holds the best iterate */
  COARSE_ERR_BREAKDOWN = -5,     /* Krylov breakdown that could not be recovered */
  COARSE_ERR_NONFINITE = -6,     /* NaN/Inf met in the data or the iteration */
  COARSE_ERR_TIMEOUT = -7,       /* a bounded device-side wait ran out */
  COARSE_ERR_NOT_GAMMA5 = -8     /* blocks violate sigma3 D_c sigma3 = D_c^H */
} coarse_status;

/* Arithmetic of a coarse apply or of the inner solver. */
typedef enum {
  COARSE_PREC_FP64 = 0, /* FP64 blocks, complex128 vectors, FP64 accumulation */
  COARSE_PREC_FP32 = 1, /* FP32 blocks, complex64 vectors, FP32 accumulation */
  COARSE_PREC_BF16 = 2  /* BF16 blocks, complex64 vectors, FP32 accumulation */
} coarse_precision;

#define COARSE_ASSUME_GAMMA5 0x1u /* hop_blocks holds only the 4 forward hops */

typedef struct {
  int32_t dims[4];      /* coarse lattice extents, each >= 2 */
  int32_t nv;           /* test vectors per chirality: n = 2*nv, nv in {8, 16, 24} */
  double mu;            /* twisted mass: D_c gets + i*mu*sigma3 on the diagonal (0 = Wilson-clover) */
  uint32_t flags;       /* COARSE_ASSUME_GAMMA5 or 0 */
  int32_t max_nrhs;     /* largest nrhs later passed to coarse_apply / coarse_solve (>= 1) */
  uint32_t precisions;  /* bit mask of (1u << coarse_precision) block copies to keep; FP64 always kept */
} coarse_op_desc;

/*
 * coarse_op_create -- ingest the Galerkin blocks of D_c = P^H D P.
 *
 * Sec. 2.2 (aggregation-based AMG; coarsest-level structure): D_c couples
 * each coarse site to itself through a dense n x n block and to its 8 nearest
 * neighbours.  Sec. 4.2 (Q = Gamma5 D is Hermitian) implies, on the coarse
 * level, sigma3 D_c sigma3 = D_c^H, so the backward hop blocks are
 * D_c[x, x-mu] = sigma3 D_c[x-mu, x]^H sigma3 and only the self block and the
 * 4 forward hops are stored ("gamma5-compressed": 5 blocks per site).
 *
 * self_blocks : device, complex128 [V][n][n], row-major; A_x (without i*mu*sigma3).
 * hop_blocks  : device, complex128 [V][8][n][n] (or [V][4][n][n] with
 *               COARSE_ASSUME_GAMMA5); hop[x][d] = D_c[x, x+mu_d] for d < 4 and
 *               D_c[x, x-mu_{d-4}] for d >= 4.
 * Without COARSE_ASSUME_GAMMA5 the backward hops and the self blocks are
 * checked against the sigma3 relation (relative defect <= 1e-10 of the
 * largest block entry) and COARSE_ERR_NOT_GAMMA5 is returned if it fails.
 * The caller keeps ownership of its buffers and may free them after return
 * (the call synchronises `stream`).  *out receives a new handle owned by the
 * caller, released with coarse_op_destroy.
 */
int coarse_op_create(const coarse_op_desc* desc, const void* self_blocks, const void* hop_blocks,
                     void* stream, coarse_op** out);

/*
 * coarse_op_update -- new block values, same shape and flags (Sec. 3.6: when
 * the multigrid setup changes the coarsest matrix, the polynomial and the
 * recycle space are rebuilt at the next solve).  Invalidates both.
 */
int coarse_op_update(coarse_op* op, const void* self_blocks, const void* hop_blocks, void* stream);

/* Releases the handle and all device memory it owns (synchronises the device). */
void coarse_op_destroy(coarse_op* op);

/*
 * coarse_apply -- y = D_c x (Sec. 2.2, the coarse nearest-neighbour stencil):
 *   y_x = (A_x + i mu sigma3) x_x + sum_mu D_c[x,x+mu] x_{x+mu} + sum_mu D_c[x,x-mu] x_{x-mu}.
 * x, y : device, [nrhs][V][n], complex128 for COARSE_PREC_FP64 and complex64
 *        otherwise; x and y must not overlap.
 * nrhs : 1 .. desc.max_nrhs.  nrhs > 1 with COARSE_PREC_BF16 runs a
 *        tensor-core multi-right-hand-side kernel (the columns rounded to BF16,
 *        FP32 accumulation): for n = 16 mma.sync on passes of up to 12 columns;
 *        for n = 32 and 48 passes of up to 16 columns, each run by mma.sync (up
 *        to 12 columns) or tcgen05.mma with tensor-memory accumulators,
 *        whichever the autotuner timed faster for the shape.  An operator created with
 *        BF16 blocks and max_nrhs > 1 keeps two more BF16 copies of its blocks
 *        (one per kernel's operand layout).
 * Asynchronous on `stream`.  The requested precision must have been enabled
 * in desc.precisions (FP64 is always available).  The FP32 / BF16 kernels
 * stage data through shared memory with bounded waits; if one ran out, that
 * launch's y is incomplete and the next synchronising call on the operator
 * (coarse_residual, coarse_solve, coarse_solve_adjoint, coarse_solve_batched)
 * returns COARSE_ERR_TIMEOUT and clears the condition.
 */
int coarse_apply(const coarse_op* op, const void* x, void* y, int nrhs, int precision, void* stream);

/* coarse_apply_adjoint -- y = D_c^H x, computed as sigma3 D_c(-mu) sigma3 x. Same arguments. */
int coarse_apply_adjoint(const coarse_op* op, const void* x, void* y, int nrhs, int precision, void* stream);

/*
 * coarse_schur_apply -- y = S x with S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe, the odd-even
 * reduced coarse operator with block-Jacobi left preconditioning (Sec. 2, Sec. 3.2),
 * applied in factored form (two passes over the lattice, each hop block read once
 * per pass, the diagonal-block inverses applied explicitly).
 * x, y : device [V/2][n] on the even sites in increasing site order (site parity =
 *        (x0 + x1 + x2 + x3) mod 2), complex128 for FP64, complex64 otherwise; no overlap.
 * Needs even lattice extents.  Asynchronous, except that the first call (and the
 * first after coarse_op_update) computes the inverses and synchronises `stream`.
 * The staged layouts of the half apply wait on their copies with bounded waits; if
 * one ran out, y is incomplete and the next synchronising call on the operator
 * returns COARSE_ERR_TIMEOUT, as for coarse_apply.
 */
int coarse_schur_apply(coarse_op* op, const void* x, void* y, int precision, void* stream);

/*
 * coarse_residual -- r = b - D_c x in FP64 and the norms ||r||_2, ||b||_2.
 * b, x, r : device complex128 [V][n] (one right-hand side); r may alias neither.
 * norms_host : host double[2] receiving (||r||, ||b||); the call synchronises `stream`.
 * The true residual that the solver's tolerance refers to.
 */
int coarse_residual(const coarse_op* op, const void* b, const void* x, void* r, double* norms_host,
                    void* stream);

/*
 * coarse_residual_noalloc -- the same result as coarse_residual (r = b - D_c x in
 * FP64, and ||r||, ||b|| into norms_host[2]), for callers that cannot allocate
 * device memory during the call: a runtime whose device memory is owned by an
 * outside pool or arena, or a code path where allocating would block or is not
 * permitted.  It calls no cudaMalloc, cudaFree or allocating library routine.
 * Instead of the operator's own work memory, all of its scratch (stencil pulls,
 * pushes and arrival counters, reduction partials) lives in one static device
 * array of about 10.5 MB that every device loading the library holds until exit.
 * The paper has no counterpart of this call.
 * Limit: V*n <= 131072 unknowns; larger operators get COARSE_ERR_INVALID_ARG.
 * The array is looked up once per device (cudaGetSymbolAddress) on the first
 * call made with that device current, and that first call also writes the
 * array's constant part with a synchronous copy: make it before any stream
 * capture.  The call itself reads its result back and synchronises `stream`, so
 * it must never be issued while `stream` is being captured; it then returns
 * COARSE_ERR_INVALID_ARG.  Every call shares the array, which keeps the previous
 * call's contents (the counters that must start at zero are cleared at the start
 * of each call): calls that overlap on the GPU, from any stream or thread, race
 * and must not be issued.  COARSE_ERR_TIMEOUT if a bounded wait of a staged
 * stencil kernel ran out during the call (r is then incomplete).
 */
int coarse_residual_noalloc(const coarse_op* op, const void* b, const void* x, void* r, double* norms_host,
                            void* stream);

/* Flags of coarse_solve_params.flags */
#define COARSE_ZERO_GUESS 0x1u      /* ignore the incoming x, start from 0 */
#define COARSE_REBUILD_POLY 0x2u    /* recompute the polynomial before this solve */
#define COARSE_RESET_RECYCLE 0x4u   /* drop the GCRO-DR recycle space before this solve */
#define COARSE_TIME_APPLY 0x8u      /* time every inner-precision stencil launch with CUDA events */
/* Evaluate the polynomial preconditioner q (Sec. 3.3) with the operator's BF16 blocks (FP32
 * vectors and accumulation) while the Krylov operator itself keeps the inner-precision blocks.
 * q(BF16 blocks) is still one fixed linear operator, so right-preconditioned GMRES and the
 * GCRO-DR recycle space (built for that operator; rebuilt when the choice changes) stay exact;
 * only the preconditioner's quality changes, by the 2^-9 block rounding.  Takes effect for
 * precision COARSE_PREC_FP32 on operators created with BF16 enabled (coarse_solve_batched: when
 * every operator has them); ignored otherwise.  The paper has no counterpart (its coarsest
 * level is single precision). */
#define COARSE_POLY_BF16 0x10u
/* Solve through the odd-even reduced system with block-Jacobi left preconditioning
 * (Sec. 2 and Sec. 3.2): the inner solver (GMRES / polynomial / GCRO-DR) works on
 * S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe over the even sites, with right-hand side
 * D_ee^{-1} (r_e - D_eo D_oo^{-1} r_o), and the odd sites are retrieved as
 * D_oo^{-1} (r_o - D_oe e_e); the FP64 refinement around it keeps the full operator.
 * Needs even lattice extents (COARSE_ERR_INVALID_ARG otherwise); FP64 solves keep the full
 * operator; coarse_solve_batched reduces every solve (all operators need even extents; the
 * BF16 inner precision then uses the single-column stencil instead of the tensor-core
 * multi-right-hand-side one); coarse_solve_adjoint reduces the adjoint
 * system sigma3 D_c(-mu) sigma3 the same way.  The first use (per sign of mu) computes the
 * inverses of the diagonal blocks A_x + i mu sigma3 in FP64. */
#define COARSE_ODD_EVEN 0x20u
/* GCRO-DR (Sec. 3.4) builds its first recycle space from the harmonic Ritz vectors of a plain
 * GMRES(m) cycle, which needs more than k Arnoldi steps.  With this flag, while the solver holds no
 * recycle space (and defl_k > 0), every cycle runs all m steps instead of ending when its
 * least-squares residual reaches the inner target, so that the first cycle yields k vectors even
 * when the system would converge sooner; the extra steps only refine that cycle's correction.
 * Meant for a setup solve; later solves reuse the space without the flag. */
#define COARSE_RECYCLE_FULL_CYCLE 0x40u
/* Latency-1 pipelined Arnoldi (Sec. 3.5, Alg. "pipe1fgmres" / "pipe1gcrodr", shifts sigma = 0):
 * the basis carries v^a_i = A v_i, so that the stencil of step i (A v^a_{i-1}) and the step's one
 * fused reduction ([C, V]^H v^a_{i-1} and ||v^a_{i-1}||^2) are independent and run concurrently on
 * two streams; h_{i,i-1} = sqrt(||v^a||^2 - sum |h|^2 - sum |b|^2) replaces the second reduction,
 * and both recurrences (v, v^a) share the coefficients.  A negative value (loss of orthogonality)
 * is a breakdown: the cycle ends with the steps before it, the next cycle restarts from the
 * residual (coarse_solve_info.breakdowns counts them).  Orthogonality can also be lost while the
 * value stays positive; a refinement step whose true FP64 residual did not decrease is undone
 * and the solve continues with classical cycles (counted as a breakdown too).  Every cycle of plain (pp-)GMRES is
 * pipelined; GCRO-DR's first cycle, without a recycle space, stays the classical GMRES cycle, and
 * each pipelined GCRO-DR cycle needs the k products A c_j of the recycle vectors (computed once per
 * recycle space).  Costs m + 1 + 2k extra vectors of storage. */
#define COARSE_PIPELINED 0x80u

typedef struct {
  int32_t m;               /* restart length of GMRES / GCRO-DR (Sec. 3.1), 2 .. 64 */
  int32_t max_restarts;    /* cycles allowed per inner solve */
  double tol;              /* target ||b - D_c x||_2 / ||b||_2, true FP64 residual */
  int32_t poly_degree;     /* d: number of Leja-ordered harmonic Ritz roots, q has degree d-1 (Sec. 3.3); 0 = off */
  int32_t defl_k;          /* k recycled harmonic Ritz vectors (Sec. 3.4); 0 = plain (pp-)GMRES; k < m */
  int32_t recycle_updates; /* u: recycle-space updates allowed, then frozen (Sec. 4.1.1) */
  int32_t precision;       /* coarse_precision of the inner solver; FP64 = no refinement */
  double inner_tol;        /* relative residual target of each inner solve (FP32/BF16 only) */
  int32_t max_ir;          /* FP64 iterative-refinement steps allowed */
  uint32_t flags;          /* COARSE_ZERO_GUESS | COARSE_REBUILD_POLY | COARSE_RESET_RECYCLE |
                              COARSE_TIME_APPLY | COARSE_POLY_BF16 | COARSE_ODD_EVEN |
                              COARSE_RECYCLE_FULL_CYCLE | COARSE_PIPELINED */
  uint64_t seed;           /* seeds the polynomial start vector when poly_start is NULL */
  const void* poly_start;  /* optional device complex128 [V][n]: start vector of the polynomial's Arnoldi */
} coarse_solve_params;

typedef struct {
  int32_t status;          /* coarse_status of this solve */
  int32_t iterations;      /* Arnoldi steps, all refinement steps together */
  int32_t matvecs;         /* applications of D_c in the inner precision */
  int32_t cycles;          /* GMRES / GCRO-DR cycles */
  int32_t ir_steps;        /* FP64 refinement steps */
  int32_t recycle_updates; /* updates of U_k, C_k made so far on this operator */
  double rel_residual;     /* true FP64 ||b - D_c x|| / ||b|| at exit */
  double setup_ms;         /* polynomial construction during this call (0 if reused) */
  double solve_ms;         /* wall time of the call */
  double apply_ms;         /* device time of the inner-precision stencil launches (COARSE_TIME_APPLY) */
  int32_t apply_count;     /* stencil launches timed in apply_ms */
  int32_t kernel_launches; /* kernels this call launched */
  double apply_bytes;      /* algorithmic bytes of the stencil launches timed in apply_ms
                              (5 n^2 V block bytes + 2 N vector bytes each, by their precision;
                              odd-even S applies: 9 n^2 V block bytes + 2.5 (V n) vector bytes) */
  double apply_ms_prec[3];    /* apply_ms split by the block precision of the launch (coarse_precision) */
  double apply_bytes_prec[3]; /* apply_bytes, split the same way */
  int32_t apply_count_prec[3];/* apply_count, split the same way */
  int32_t breakdowns;         /* pipelined cycles ended by a negative h^2 (COARSE_PIPELINED) */
} coarse_solve_info;

/*
 * coarse_solve -- solve D_c x = b (Sec. 3.6, the whole coarsest-level solver):
 * restarted GMRES(m) (Sec. 3.1) with right polynomial preconditioner
 * q(D_c) built from Leja-ordered harmonic Ritz values (Sec. 3.3, Alg. 3) and
 * GCRO-DR deflation by k harmonic Ritz vectors with recycling across restarts
 * and right-hand sides (Sec. 3.4), inside FP64 iterative refinement when the
 * inner precision is FP32 or BF16.
 * b : device complex128 [nrhs][V][n];  x : device complex128 [nrhs][V][n],
 *     initial guess (unless COARSE_ZERO_GUESS) and result.  The right-hand
 *     sides are solved one after another and share the polynomial and the
 *     recycle space, which the handle keeps for later calls.
 * info_host : host array of nrhs records (may be NULL).
 * Synchronises `stream`.  Returns COARSE_ERR_NOT_CONVERGED if any column
 * missed tol (x then holds the best iterate).
 */
int coarse_solve(coarse_op* op, const void* b, void* x, int nrhs, const coarse_solve_params* params,
                 coarse_solve_info* info_host, void* stream);

/*
 * coarse_solve_adjoint -- solve D_c^H lambda = c via D_c^H = sigma3 D_c(-mu) sigma3
 * (coarse form of Gamma5-hermiticity, Sec. 4.2): lambda = sigma3 D_c(-mu)^{-1} sigma3 c.
 * Same arguments as coarse_solve (b = c, x = lambda).  For mu = 0 it shares the
 * polynomial and the recycle space of the forward solve.
 */
int coarse_solve_adjoint(coarse_op* op, const void* b, void* x, int nrhs, const coarse_solve_params* params,
                         coarse_solve_info* info_host, void* stream);

/*
 * coarse_solve_batched -- nops independent solves (operators of uneven size),
 * advanced together: every Krylov phase of all unfinished solves runs in one
 * kernel launch, and the whole lockstep solve (all refinement steps, cycles and
 * Arnoldi steps) is one CUDA graph, launched once, whose nested conditional WHILE
 * nodes are driven by control kernels on the device (bounded by max_ir,
 * max_restarts and m).  ops[i], b[i], x[i], nrhs[i] as in coarse_solve; all
 * operators use the same params.  infos: host array of sum(nrhs) records in
 * (operator, column) order.  Synchronises `stream`.
 * Each solve follows Sec. 3.6 exactly as coarse_solve does (restarted GMRES,
 * polynomial of Sec. 3.3, GCRO-DR of Sec. 3.4, FP64 refinement); the batching
 * itself has no counterpart in the paper, which solves one coarsest system at a
 * time, distributed over many processes.
 */
int coarse_solve_batched(coarse_op* const* ops, int nops, const void* const* b, void* const* x,
                         const int* nrhs, const coarse_solve_params* params, coarse_solve_info* infos,
                         void* stream);

/*
 * coarse_block_grad -- block gradients of a real loss L through x = D_c^{-1} b
 * given lambda = D_c^{-H} dL/dx*:  G_self[x] = -lambda_x x_x^H and
 * G_hop[x][d] = -lambda_x x_{x +- mu_d}^H (convention dL = Re sum conj(G) dD).
 * The paper has no counterpart (it never differentiates the coarse solve); the
 * adjoint solve that provides lambda uses D_c^H = sigma3 D_c(-mu) sigma3, the
 * coarse form of the Gamma5-hermiticity of Sec. 4.2.
 * lambda, x : device complex128 [V][n];  g_self : device complex128 [V][n][n].
 * hop_dirs  : 8 -> g_hop is [V][8][n][n] (canonical 9-block layout, every hop block an
 *             independent input);  4 -> g_hop is [V][4][n][n], the gradient with respect to
 *             the forward blocks of a COARSE_ASSUME_GAMMA5 input, whose backward hops
 *             sigma3 F^H sigma3 are derived from them: the backward-hop gradient of x + mu is
 *             folded onto F_{x,mu} as sigma3 G^H sigma3.
 * Asynchronous on `stream`.
 */
int coarse_block_grad(const coarse_op* op, const void* lambda, const void* x, void* g_self, void* g_hop,
                      int hop_dirs, void* stream);

/*
 * coarse_op_poly -- the Leja-ordered harmonic Ritz values theta_1..theta_d
 * (Sec. 3.3, Alg. 2) currently held for `precision`.  theta_host: host double[2*cap]
 * (re, im pairs); *d receives the degree (0 if none is built).
 */
int coarse_op_poly(const coarse_op* op, int precision, double* theta_host, int cap, int* d);

/*
 * coarse_autotune_report -- the launch autotuner's decisions as text, one line per
 * kernel family and shape: "<key> -> <config> <microseconds> | <candidates timed>".
 * The paper has no counterpart: its kernels have a fixed launch shape.  The first
 * call of a kernel for a new shape times each candidate configuration on the
 * caller's stream (synchronising it) and keeps the fastest; a stream that is being
 * captured into a CUDA graph is never timed (the default configuration runs).  If
 * the environment variable COARSE_AUTOTUNE_CACHE names a file, decisions are read
 * from it at first use and new ones appended.
 * buf : host char[len]; receives a NUL-terminated (possibly truncated) report.
 */
int coarse_autotune_report(char* buf, long long len);

/*
 * coarse_autotune_set -- fixes the launch configuration for one kernel family and shape
 * instead of timing the candidates, e.g. to reproduce a measurement or a result bit for bit
 * across processes.  key: a key as coarse_autotune_report prints it ("eo/p1/n48/v15"), with or
 * without its GPU-model suffix ("@sm103x152"); without it the decision applies to every device.
 * (a, b, c): the configuration, as in the report; a < 0 forgets the decision instead, so that
 * the next launch times the candidates again.  Takes effect from the next launch.  The paper
 * has no counterpart.
 */
int coarse_autotune_set(const char* key, int a, int b, int c);

/*
 * coarse_recycle_check -- re-evaluates the GCRO-DR recycle space that the handle holds for one
 * inner system (Sec. 3.4: U_k, C_k with A U_k = C_k and C_k^H C_k = I, where A = D q(D) is the
 * right-preconditioned operator of the solves that built it, Sec. 3.3).  One application of A per
 * column, polynomial chain included, in the inner precision of those solves.
 * precision : inner precision of the solves (coarse_precision).
 * odd_even  : 0 = the full-operator system, 1 = the odd-even reduced system (COARSE_ODD_EVEN),
 *             where D stands for S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe.
 * adjoint   : 1 = the system of coarse_solve_adjoint (the same as the forward one when mu = 0).
 * out_host  : host double[4] receiving max_i ||A u_i - c_i|| / ||c_i||, max_ij |(C^H C - I)_ij|,
 *             k (columns held; 0 and zero defects if no recycle space was formed) and the number
 *             of recycle-space updates made.
 * Synchronises `stream`; uses the solver's own work vectors (do not overlap it with a solve on the
 * same handle).
 */
int coarse_recycle_check(coarse_op* op, int precision, int odd_even, int adjoint, double* out_host, void* stream);

/*
 * coarse_recycle_get -- copies out the recycle space named as in coarse_recycle_check
 * (Sec. 3.4: U_k and C_k = A U_k, C_k^H C_k = I), e.g. to inspect it or to keep it with a
 * checkpoint of the multigrid setup.
 * u, c : device buffers of cap columns each, [cap][N] complex128 for FP64 solves and complex64
 *        otherwise, N = V n (full operator) or V n / 2 (odd-even reduced system, even sites in
 *        increasing site order).  Only the first *k columns are written.
 * *k   : receives the number of columns held (0: none, and u, c may then be NULL).
 * Returns COARSE_ERR_INVALID_ARG if cap is below the number held.  Synchronises `stream`.
 */
int coarse_recycle_get(coarse_op* op, int precision, int odd_even, int adjoint, void* u, void* c, int cap, int* k,
                       void* stream);

/*
 * coarse_measure_fp64_fma -- FP64 FMA throughput of the current device in TFLOP/s, from a plain
 * loop of independent FMA chains (8 CTAs of 256 threads per SM, `iters` FMAs per chain, best of
 * three timed launches on `stream`, which it synchronises).  The FP64 stencil that computes the
 * refinement residual is bound by this rate on GB300, and this is the peak its roofline uses.
 * The paper has no counterpart.
 */
int coarse_measure_fp64_fma(int iters, double* tflops_host, void* stream);

/*
 * coarse_recycle_set -- installs a recycle space (U_k, C_k; Sec. 3.4) for the system named as in
 * coarse_recycle_check, e.g. one saved with coarse_recycle_get, so that later solves deflate
 * with it from their first cycle.  The space must belong to the right-preconditioned operator
 * A = D q(D) that the solver currently holds (same polynomial) and satisfy A U_k = C_k,
 * C_k^H C_k = I; nothing checks this (coarse_recycle_check measures it afterwards).
 * u, c    : device [k][N] as for coarse_recycle_get (copied; the caller keeps ownership).
 * k       : columns; 0 drops the recycle space.
 * updates : the solver's count of updates made, compared with recycle_updates of later solves
 *           (>= recycle_updates keeps the space frozen).
 * The handle must already hold a solver of that system created with defl_k >= k (one solve with
 * those parameters); COARSE_ERR_INVALID_ARG otherwise.  Synchronises `stream`.
 */
int coarse_recycle_set(coarse_op* op, int precision, int odd_even, int adjoint, const void* u, const void* c, int k,
                       int updates, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* coarse_last_error(void);

/* Library version string. */
const char* coarse_version(void);

#ifdef __cplusplus
}
#endif

#endif /* COARSE_H */
