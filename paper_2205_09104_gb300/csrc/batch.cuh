// Batched lockstep engine: descriptors of the solves that advance together and the
// launchers of the batched kernels.  One solve = one right-hand-side column of one
// operator; all solves of a batch run the same phase sequence, each phase is one kernel
// launch over all solves (work items mapped to solves through prefix sums), and the
// per-solve stop / active flags on the device skip solves that are finished.
#pragma once

#include "common.cuh"
#include "solver_state.cuh"

namespace coarse {

constexpr int kBatchMaxQ = 104;  // dots per reduction (equals the chunked kernels' limit)

struct BSolve {
  // operator (shared by the solves of one operator)
  const void* blk;     // inner-precision blocks [V][5][n][n]
  const void* blk_poly; // blocks of the polynomial-chain phases (BF16 with COARSE_POLY_BF16, else blk)
  const void* blk64;   // FP64 blocks
  const int* nb;       // [V][8]
  int V, n, N;
  int kc;              // recycle vectors in use (frozen)
  double mu;
  // stencil scratch of this solve (pull partials, pushes, arrival counters + error flag)
  void* part;
  void* push;
  int* cnt;
  // vectors of the inner precision (complex64)
  void** vt;           // [m + 1] Krylov basis
  void** qt;           // [kc + m + 1]: C_k then the basis
  void** ut;           // [kc + m]: U_k then the basis
  void* r;
  void* e;
  void* t;
  void* sa;
  void* sb;
  void* acc;
  // FP64 refinement
  const double2* b64;
  double2* x64;
  double2* r64;
  void* part64;        // FP64 stencil scratch
  // polynomial chain coefficients (3 per chain step, padded to the batch degree)
  const double2* polyc;
  // dense state
  CycleState* st;
  Dense dn;
  double2* h1;
  double2* h2;
  double* partial;     // reduction partials of this solve
  unsigned* counter;   // last-CTA counter of this solve
  double* norm2;       // [0] ||r||^2 (inner), [1] ||r64||^2, [2] ||b||^2
  int* flags;          // [0] inner-active this cycle, [1] done (tolerance met)
  int nch;             // CTAs of this solve in the chunked reductions
  // odd-even reduction (COARSE_ODD_EVEN): the Krylov vectors above are the even halves (N = V n / 2);
  // the FP64 refinement keeps full-length vectors (Nf = V n, nchf chunks)
  int eo;
  int Nf, nchf;
  const void* inv;      // inverses of the diagonal blocks in the inner precision [V][n][n]
  const void* inv_poly; // the same in the precision of the polynomial-chain phases
  const int4* eo_rec;   // neighbour records (coarse_op::eo_rec)
  const int* eo_sites;  // even sites, then odd sites, increasing (coarse_op::eo_sites)
  void* f32;            // full-length FP32 work vector (residual in, correction out)
  void* re;             // even / odd halves of the residual
  void* ro;
  void* to;             // D_oo^{-1} r_o
  void* eoe;            // odd part of the correction
  void* todd;           // odd intermediate of an S apply
};

// Which vector a batched stencil phase reads / writes.
enum BSel : int { BS_NONE = -1, BS_VJ = 0, BS_VJ1, BS_SA, BS_SB, BS_ACC, BS_T, BS_R, BS_E, BS_TODD, BS_RE, BS_RO,
                  BS_TO, BS_EOE };

// Gate of a batched phase: run the solve's part only if ...
enum BGate : int {
  BG_STEP = 0,   // ... its Arnoldi cycle is running (st->stop == 0)
  BG_ACTIVE = 1, // ... it is inner-active this cycle (flags[0])
  BG_TAIL = 2,   // ... it is inner-active and its cycle made at least one step
  BG_NOTDONE = 3 // ... it has not met the tolerance (flags[1] == 0)
};

struct BApply {
  const BSolve* S;
  const int* sidx;      // solves of this n-group
  const int* site_off;  // prefix sums of their site counts (count + 1 entries)
  int count;
  int total;            // total sites
  int mode;             // ApplyMode
  int xsel, ysel;       // BSel
  int coef_off;         // offset (in double2) into polyc for POLY modes
  int gate;             // BGate
  const int* step;      // device step counter
  int poly_blocks;      // 1: the solves' blk_poly (polynomial-chain phases), 0: blk
};

// work item -> solve, gates and vector selection shared by the batched kernels
__device__ inline int find_solve(const int* off, int count, int g) {
  int lo = 0, hi = count;  // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ inline bool bgate(const BSolve& s, int gate) {
  switch (gate) {
    case BG_STEP: return s.st->stop == 0;
    case BG_ACTIVE: return s.flags[0] != 0;
    case BG_TAIL: return s.flags[0] != 0 && s.st->j > 0;
    case BG_NOTDONE: return s.flags[1] == 0;
  }
  return false;
}

__device__ inline void* bsel(const BSolve& s, int sel, int step) {
  switch (sel) {
    case BS_VJ: return s.vt[step];
    case BS_VJ1: return s.vt[step + 1];
    case BS_SA: return s.sa;
    case BS_SB: return s.sb;
    case BS_ACC: return s.acc;
    case BS_T: return s.t;
    case BS_R: return s.r;
    case BS_E: return s.e;
    case BS_TODD: return s.todd;
    case BS_RE: return s.re;
    case BS_RO: return s.ro;
    case BS_TO: return s.to;
    case BS_EOE: return s.eoe;
  }
  return nullptr;
}

// One batched half apply of the odd-even reduced operator (Sec. 2, Sec. 3.2) over an n-group:
// output sites of parity out_par, y = B^{-1} (z - sum hops v) or base - B^{-1} (...), chain epilogue.
struct BEoApply {
  const BSolve* S;
  const int* sidx;      // solves of this n-group
  const int* site_off;  // prefix sums of their half-site counts V / 2 (count + 1 entries)
  int count;
  int total;            // total output sites
  int out_par;
  int vsel, zsel, bsel, ysel;  // BSel (BS_NONE: absent)
  int mode;
  int coef_off;
  int gate;
  const int* step;
  int poly_blocks;      // 1: the chain's blocks and inverses
};
int launch_beo_half(int prec, int n, const BEoApply& b, cudaStream_t s);

int launch_bapply(int prec, int n, const BApply& a, cudaStream_t s);

// ---- multi-RHS (tensor-core) stencil phases: every column of one operator in one pass
struct BMOp {
  const void* frag;    // fragment-native BF16 blocks (coarse_op::mrhs)
  const int* nb;
  void* xb;            // packed BF16 B fragments of the phase's input columns, [V][T][NT][32] uint2
  int V, n, R, T;      // sites, dof per site, columns (solves), column tiles ceil(R/4)
  int s0;              // first solve of the operator (its columns are s0 .. s0 + R - 1)
  float mu;
};

struct BMApply {
  const BSolve* S;
  const BMOp* ops;
  const int* idx;       // operators of this n-group (count)
  const int* grp_off;   // prefix sums of their site groups of P sites (count + 1)
  const int* grp_op;    // position in idx of the operator of each site group (total_groups)
  int count;
  int total_groups;
  int mode, xsel, ysel, coef_off, gate;
  const int* step;
  int* err;             // raised if a bounded wait of the pipeline expired
};

// packs the input columns (BSel xsel, gated) of all operators; word_off = prefix sums over the
// operators of their packed words (nops + 1 entries)
int launch_bpack_mrhs(const BMApply& a, int nops, const int* word_off, int total_words, cudaStream_t s);
// the stencil phase of one n-group; P sites per stage, S stages
int launch_bapply_mrhs(int n, int P, int S, const BMApply& a, cudaStream_t s);
int launch_bapply64_residual(int n, const BApply& a, cudaStream_t s);

// chunked Gram-Schmidt / vector phases over all solves
enum BVecOp : int {
  BV_CGS_DOT = 0,    // h1 = Q^H V[j+1]                    (gate step)
  BV_CGS_UPDDOT,     // V[j+1] -= Q h1 ; h2 = Q^H V[j+1]      (gate step)
  BV_CGS_UPDNORM,    // V[j+1] -= Q h2 ; st->wnorm2           (gate step)
  BV_PROJ_DOT,       // ycoef = C^H r                         (gate active, kc > 0)
  BV_PROJ_UPD,       // r -= C ycoef ; norm2[0]               (gate active)
  BV_RES_UPD,        // r -= V[0..j] z ; norm2[0]             (gate tail)
  BV_NORM_R,         // norm2[0] = ||r||^2                     (gate active)
};
int launch_bvec(int op, const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E,
                const int* step, cudaStream_t s);

// per-solve elementwise phases
enum BElem : int {
  BE_NORMALIZE = 0,  // V[j+1] *= inv_h if the finalize of step j ran
  BE_START,          // V[0] = r * inv_h                       (gate step)
  BE_COMBINE_T,      // t = ut[0..kc+j) . ycoef                (gate tail)
  BE_COMBINE_U,      // t = U_k . ycoef[0..kc)                 (gate active, kc > 0)
  BE_AXPY_E,         // e += acc                                (gate tail / active)
  BE_AXPY_E_PROJ,    // e += acc after the projection          (gate active, kc > 0)
  BE_TO_LOW,         // r = r64 / ||r64||, e = 0                (gate not done)
  BE_ADD_LOW,        // x64 += ||r64|| e                        (gate not done)
  BE_ZERO_X,         // x64 = 0                                 (all)
  // odd-even reduction (Sec. 2): the refinement's residual and correction through the halves
  BE_TO_LOW_F,       // f32 = r64 / ||r64||                     (gate not done, full length)
  BE_EO_SPLIT,       // re, ro = even / odd parts of f32, e = 0 (gate not done, half length)
  BE_EO_MERGE,       // f32 = (e on the even sites, eoe on the odd sites) (gate not done, half length)
  BE_ADD_LOW_F,      // x64 += ||r64|| f32                      (gate not done, full length)
};
// Phases over the full-length vectors (launched with the full-length chunk table): the FP64
// refinement's and those that read or write r64, x64 or f32.
__host__ __device__ inline bool belem_full(int op) {
  return op == BE_TO_LOW || op == BE_ADD_LOW || op == BE_ZERO_X || op == BE_TO_LOW_F || op == BE_ADD_LOW_F;
}
// aux: source of BE_AXPY_E (BS_ACC or BS_T); gate: BGate of BE_AXPY_E
int launch_belem(int op, const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E,
                 const int* step, int aux, int gate, cudaStream_t s);

// per-solve dense kernels (one CTA per solve)
int launch_bcycle_init(const BSolve* S, int nsolves, int m, double target, cudaStream_t s);
int launch_bfinalize(const BSolve* S, int nsolves, cudaStream_t s);
int launch_bcycle_solve(const BSolve* S, int nsolves, cudaStream_t s);
// which = 1: norm2[1] = ||r64||^2, which = 2: norm2[2] = ||b64||^2
int launch_bnorms64(const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E, int which,
                    cudaStream_t s);
int batch_chunk_elems(int maxN);     // elements per lane of the chunked kernels for the largest solve
int batch_chunks(int N, int E);      // CTAs of one solve
int launch_step_inc(int* step, cudaStream_t s);

}  // namespace coarse
