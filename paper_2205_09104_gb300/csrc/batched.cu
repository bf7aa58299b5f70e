// coarse_solve_batched: many independent solves of uneven operators advanced in lockstep.
//
// Every (operator, right-hand-side column) is one solve.  Setup (polynomial and the first
// u recycle-space updates) runs per operator through the single-operator solver; the solves
// then share their operator's blocks, polynomial and frozen U_k, C_k.  In the lockstep phase
// each Krylov phase is ONE kernel launch over all solves (per n-group for the stencil), and
// per-solve stop / active / done flags on the device skip the solves that are finished.  The
// whole lockstep solve -- every refinement step, cycle and Arnoldi step -- is one CUDA graph
// launched once: three nested conditional WHILE nodes whose conditions control kernels set on
// the device (with iteration bounds), so the host waits only for the end of the batch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "mrhs_core.cuh"
#include "oddeven.cuh"
#include "solver.cuh"

namespace coarse {
namespace {

#define TRY(call)                     \
  do {                                \
    int _rc = (call);                 \
    if (_rc != COARSE_OK) return _rc; \
  } while (0)

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Group {
  int n = 0;
  int count = 0;
  int total = 0;
  int* sidx = nullptr;
  int* site_off = nullptr;
};

// n-group of the multi-RHS stencil phases
struct MGroup {
  int n = 0, P = 1, S = 3;
  BMApply a{};  // operator list, site-group offsets (device); phase fields filled per launch
};

// sites per stage and pipeline stages of the batched multi-RHS kernel per n (the standalone
// kernel's autotuned choices on 4^4 .. 8^4 lattices)
inline void bm_shape(int n, int* P, int* S) {
  *P = n == 48 ? 1 : 2;
  *S = n == 16 ? 5 : 3;
}

struct Batch {
  int prec = COARSE_PREC_FP32;
  int poly_prec = COARSE_PREC_FP32;  // blocks of the polynomial-chain phases
  bool mrhs = false;              // BF16 stencil phases on the tensor-core multi-RHS kernel
  std::vector<MGroup> mgroups;
  BMOp* dops = nullptr;
  int nops = 0;
  int* word_off = nullptr;
  int total_words = 0;
  int* merr = nullptr;
  int m = 0, dd = 0, ns = 0, E = 4, total_chunks = 0, steps_max = 0;
  bool any_kc = false;
  char* mem = nullptr;
  BSolve* dS = nullptr;
  int* step = nullptr;
  CycleState* states = nullptr;
  double* norms = nullptr;
  int* flags = nullptr;
  int* chunk_off = nullptr;
  // odd-even reduction: the Krylov phases run on the even halves (chunk_off, total_chunks), the
  // refinement's full-length phases on chunk_off_f / total_chunks_f; egroups: half-site groups
  bool eo = false;
  int* chunk_off_f = nullptr;
  int total_chunks_f = 0;
  std::vector<Group> egroups;
  std::vector<Group> groups;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long launches = 0;

  ~Batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (mem) cudaFree(mem);
  }

  // one half apply of the odd-even reduced operator over every n-group
  int eo_half(int out_par, int vsel, int zsel, int bsel, int ysel, int mode, int coef_off, int gate, bool chain,
              cudaStream_t s) {
    for (const Group& g : egroups) {
      BEoApply a;
      a.S = dS;
      a.sidx = g.sidx;
      a.site_off = g.site_off;
      a.count = g.count;
      a.total = g.total;
      a.out_par = out_par;
      a.vsel = vsel;
      a.zsel = zsel;
      a.bsel = bsel;
      a.ysel = ysel;
      a.mode = mode;
      a.coef_off = coef_off;
      a.gate = gate;
      a.step = step;
      a.poly_blocks = chain ? 1 : 0;
      TRY(launch_beo_half(chain ? poly_prec : prec, g.n, a, s));
    }
    return COARSE_OK;
  }

  // one stencil phase over all n-groups (chain: a polynomial-chain phase, on the chain's blocks)
  int apply_phase(int mode, int xsel, int ysel, int coef_off, int gate, cudaStream_t s, bool chain = false) {
    if (eo) {
      // y = S x: t_o = B_o^{-1} D_oe x, then y = x - B_e^{-1} D_eo t_o with the chain epilogue
      TRY(eo_half(1, xsel, BS_NONE, BS_NONE, BS_TODD, APPLY_PLAIN, 0, gate, chain, s));
      return eo_half(0, BS_TODD, BS_NONE, xsel, ysel, mode, coef_off, gate, chain, s);
    }
    if (mrhs) {
      for (size_t i = 0; i < mgroups.size(); ++i) {
        BMApply a = mgroups[i].a;
        a.mode = mode;
        a.xsel = xsel;
        a.ysel = ysel;
        a.coef_off = coef_off;
        a.gate = gate;
        if (i == 0) TRY(launch_bpack_mrhs(a, nops, word_off, total_words, s));
        TRY(launch_bapply_mrhs(mgroups[i].n, mgroups[i].P, mgroups[i].S, a, s));
      }
      return COARSE_OK;
    }
    for (const Group& g : groups) {
      BApply a;
      a.S = dS;
      a.sidx = g.sidx;
      a.site_off = g.site_off;
      a.count = g.count;
      a.total = g.total;
      a.mode = mode;
      a.xsel = xsel;
      a.ysel = ysel;
      a.coef_off = coef_off;
      a.gate = gate;
      a.step = step;
      a.poly_blocks = chain ? 1 : 0;
      TRY(launch_bapply(chain ? poly_prec : prec, g.n, a, s));
    }
    return COARSE_OK;
  }

  // acc = q(A) x for every solve passing `gate` (x = BS_VJ or BS_T); returns the BSel of the result
  int precondition(int xsel, int gate, cudaStream_t s, int* result) {
    if (dd == 0) {
      *result = xsel;
      return COARSE_OK;
    }
    TRY(apply_phase(APPLY_POLY_FIRST, xsel, BS_SA, 0, gate, s, true));
    for (int i = 2; i < dd; ++i) {
      const bool even = (i % 2) == 0;
      TRY(apply_phase(APPLY_POLY, even ? BS_SA : BS_SB, even ? BS_SB : BS_SA, 3 * (i - 1), gate, s, true));
    }
    *result = BS_ACC;
    return COARSE_OK;
  }

  int vec(int op, cudaStream_t s) { return launch_bvec(op, dS, ns, chunk_off, total_chunks, E, step, s); }
  int elem(int op, cudaStream_t s, int aux = BS_ACC, int gate = BG_TAIL) {
    if (belem_full(op)) return launch_belem(op, dS, ns, chunk_off_f, total_chunks_f, E, step, aux, gate, s);
    return launch_belem(op, dS, ns, chunk_off, total_chunks, E, step, aux, gate, s);
  }
  int norms64(int which, cudaStream_t s) {
    return launch_bnorms64(dS, ns, chunk_off_f, total_chunks_f, E, which, s);
  }

  // refinement step, odd-even: the reduced right-hand side r = B_e^{-1} (r_e - D_eo D_oo^{-1} r_o)
  // from the full residual, and afterwards the full correction from e (Sec. 2, Sec. 3.2)
  int eo_rhs(cudaStream_t s) {
    TRY(elem(BE_TO_LOW_F, s));
    TRY(elem(BE_EO_SPLIT, s));
    TRY(eo_half(1, BS_NONE, BS_RO, BS_NONE, BS_TO, APPLY_PLAIN, 0, BG_NOTDONE, false, s));
    return eo_half(0, BS_TO, BS_RE, BS_NONE, BS_R, APPLY_PLAIN, 0, BG_NOTDONE, false, s);
  }
  int eo_correction(cudaStream_t s) {
    TRY(eo_half(1, BS_E, BS_NONE, BS_TO, BS_EOE, APPLY_PLAIN, 0, BG_NOTDONE, false, s));
    TRY(elem(BE_EO_MERGE, s));
    return elem(BE_ADD_LOW_F, s);
  }

  // one Arnoldi step of every running solve: A v_j -> CGS2 -> finalize -> normalise -> step++
  int step_sequence(cudaStream_t s) {
    int src = BS_VJ;
    TRY(precondition(BS_VJ, BG_STEP, s, &src));
    TRY(apply_phase(APPLY_PLAIN, src, BS_VJ1, 0, BG_STEP, s));
    TRY(vec(BV_CGS_DOT, s));
    TRY(vec(BV_CGS_UPDDOT, s));
    TRY(vec(BV_CGS_UPDNORM, s));
    TRY(launch_bfinalize(dS, ns, s));
    TRY(elem(BE_NORMALIZE, s));
    return launch_step_inc(step, s);
  }

  int residual64(cudaStream_t s) {
    for (const Group& g : groups) {
      BApply a;
      a.S = dS;
      a.sidx = g.sidx;
      a.site_off = g.site_off;
      a.count = g.count;
      a.total = g.total;
      a.mode = APPLY_AXPBY;
      a.xsel = a.ysel = 0;
      a.coef_off = 0;
      a.gate = BG_NOTDONE;
      a.step = step;
      a.poly_blocks = 0;
      TRY(launch_bapply64_residual(g.n, a, s));
    }
    return norms64(1, s);
  }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ---- device-side control of the whole batched solve (refinement steps, cycles, Arnoldi steps)
//
// The whole lockstep solve is one CUDA graph: three nested conditional WHILE nodes (refinement
// step > cycle > Arnoldi step) whose conditions are set by the control kernels below from the
// per-solve state on the device, each with its own iteration bound, so that the host launches
// the graph once and reads the per-solve results at the end.

struct BCtl {
  int ir, cyc, steps_run, cycles_run;  // loop counters (steps_run, cycles_run: totals, for accounting)
  int max_ir, max_cyc, steps_max;
  double tol, inner_tol;
  cudaGraphConditionalHandle h_ir, h_cyc, h_step;
};

struct BInfo {
  int status, iterations, cycles, ir_steps;
  double bn, rn;
};

constexpr int kCtlThreads = 1024;

__device__ int ctl_any(int v) {
  return __syncthreads_or(v);
}

// after the initial residual: ||b||, ||r||, solves already done, and the refinement loop's condition
__global__ void __launch_bounds__(kCtlThreads) kb_ctl_start(BCtl* c, const BSolve* S, BInfo* I, int ns) {
  int left = 0;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    const double* n2 = S[q].norm2;
    int* fl = S[q].flags;
    const double bn = sqrt(fmax(n2[2], 0.0)), rn = sqrt(fmax(n2[1], 0.0));
    BInfo in{};
    in.bn = bn;
    in.rn = rn;
    int done;
    if (!isfinite(bn) || !isfinite(rn)) {
      in.status = COARSE_ERR_NONFINITE;
      done = 1;
    } else {
      done = (bn == 0.0 || rn <= c->tol * bn) ? 1 : 0;
    }
    I[q] = in;
    fl[0] = 0;
    fl[1] = done;
    left |= !done;
  }
  left = ctl_any(left);
  if (threadIdx.x == 0) {
    c->ir = c->cyc = c->steps_run = c->cycles_run = 0;
    cudaGraphSetConditional(c->h_ir, (left && c->max_ir > 0) ? 1u : 0u);
  }
}

// start of a refinement step: the unfinished solves become inner-active with their inner targets
__global__ void __launch_bounds__(kCtlThreads) kb_ir_begin(BCtl* c, const BSolve* S, const BInfo* I, int ns) {
  int act = 0;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    int* fl = S[q].flags;
    const int a = !fl[1];
    fl[0] = a;
    S[q].norm2[3] = fmax(c->inner_tol, 0.5 * c->tol * I[q].bn / fmax(I[q].rn, 1e-300));
    act |= a;
  }
  act = ctl_any(act);
  if (threadIdx.x == 0) {
    c->cyc = 0;
    cudaGraphSetConditional(c->h_cyc, (act && c->max_cyc > 0) ? 1u : 0u);
  }
}

// after a cycle's start: Arnoldi steps run while some cycle runs and fewer than steps_max were taken
__global__ void __launch_bounds__(kCtlThreads) kb_step_gate(BCtl* c, const BSolve* S, const int* step, int ns,
                                                            int count_step) {
  int run = 0;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) run |= S[q].st->stop == 0;
  run = ctl_any(run);
  if (threadIdx.x == 0) {
    if (count_step) c->steps_run++;
    cudaGraphSetConditional(c->h_step, (run && *step < c->steps_max) ? 1u : 0u);
  }
}

// end of a cycle: statistics, solves that leave the inner loop, the cycle loop's condition
__global__ void __launch_bounds__(kCtlThreads) kb_cycle_end(BCtl* c, const BSolve* S, BInfo* I, int ns) {
  int act = 0;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    int* fl = S[q].flags;
    if (!fl[0]) continue;
    const CycleState& cs = *S[q].st;
    I[q].cycles++;
    I[q].iterations += cs.j;
    if (cs.status & ST_NONFINITE) {
      I[q].status = COARSE_ERR_NONFINITE;
      fl[1] = 1;
      fl[0] = 0;
      continue;
    }
    if (cs.j == 0 || cs.resid <= cs.target || (cs.status & (ST_LUCKY | ST_ZERO))) fl[0] = 0;
    act |= fl[0];
  }
  act = ctl_any(act);
  if (threadIdx.x == 0) {
    c->cyc++;
    c->cycles_run++;
    cudaGraphSetConditional(c->h_cyc, (act && c->cyc < c->max_cyc) ? 1u : 0u);
  }
}

// end of a refinement step: new true residuals, solves that met the tolerance, the loop's condition
__global__ void __launch_bounds__(kCtlThreads) kb_ir_end(BCtl* c, const BSolve* S, BInfo* I, int ns) {
  int left = 0;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    int* fl = S[q].flags;
    if (fl[1]) continue;
    I[q].ir_steps++;
    const double rn = sqrt(fmax(S[q].norm2[1], 0.0));
    I[q].rn = rn;
    if (!isfinite(rn)) {
      I[q].status = COARSE_ERR_NONFINITE;
      fl[1] = 1;
    } else if (rn <= c->tol * I[q].bn) {
      fl[1] = 1;
    }
    left |= !fl[1];
  }
  left = ctl_any(left);
  if (threadIdx.x == 0) {
    c->ir++;
    cudaGraphSetConditional(c->h_ir, (left && c->ir < c->max_ir) ? 1u : 0u);
  }
}

// Adds a WHILE node on `handle` at the capture position of `s` and returns its (empty) body.
int add_while(cudaStream_t s, cudaGraphConditionalHandle handle, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  COARSE_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd));
  if (cst != cudaStreamCaptureStatusActive) {
    set_error("coarse_solve_batched: stream is not capturing");
    return COARSE_ERR_CUDA;
  }
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = handle;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  COARSE_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  *body = prm.conditional.phGraph_out[0];
  COARSE_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return COARSE_OK;
}

// Captures fill(stream) into the body graph of a conditional node.
template <class F>
int capture_body(cudaGraph_t body, cudaStream_t cs, F&& fill) {
  COARSE_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = fill(cs);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (rc == COARSE_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture (conditional body)");
  return rc;
}

size_t graph_kernels(cudaGraph_t g) {
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  return n;
}

}  // namespace
}  // namespace coarse

using namespace coarse;

extern "C" int coarse_solve_batched(coarse_op* const* ops, int nops, const void* const* b, void* const* x,
                                    const int* nrhs, const coarse_solve_params* p, coarse_solve_info* infos,
                                    void* stream) {
  if (nops < 0 || (nops > 0 && (!ops || !b || !x || !nrhs || !p))) {
    set_error("coarse_solve_batched: NULL array or negative nops");
    return COARSE_ERR_INVALID_ARG;
  }
  if (nops == 0) return COARSE_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double t0 = now_ms();
  if (p->precision == COARSE_PREC_FP64) {
    // the lockstep engine runs FP32/BF16 inner solves; FP64 solves go one after another
    int worst = COARSE_OK;
    size_t at = 0;
    for (int i = 0; i < nops; ++i) {
      int rc = coarse_solve(ops[i], b[i], x[i], nrhs[i], p, infos ? infos + at : nullptr, stream);
      at += nrhs[i] > 0 ? nrhs[i] : 0;
      if (rc != COARSE_OK && rc != COARSE_ERR_NOT_CONVERGED) return rc;
      if (rc != COARSE_OK) worst = rc;
    }
    return worst;
  }
  for (int i = 0; i < nops; ++i) {
    if (!ops[i] || !b[i] || !x[i] || nrhs[i] < 1) {
      set_error("coarse_solve_batched: entry %d has a NULL pointer or nrhs < 1", i);
      return COARSE_ERR_INVALID_ARG;
    }
  }
  if (p->m < 2 || p->m > kMaxDense || p->defl_k < 0 || p->defl_k > kMaxK || (p->defl_k > 0 && p->defl_k >= p->m) ||
      p->poly_degree < 0 || p->poly_degree > kMaxPoly || !(p->tol > 0.0) || p->max_restarts < 1 || p->max_ir < 1 ||
      !(p->inner_tol > 0.0 && p->inner_tol < 1.0) || p->precision < 0 || p->precision > 2) {
    set_error("coarse_solve_batched: invalid solve parameters");
    return COARSE_ERR_INVALID_ARG;
  }
  const int prec = p->precision;
  const int m = p->m, k = p->defl_k, d = p->poly_degree;
  const long long launches0 = launches_so_far();
  // COARSE_ODD_EVEN: every solve's inner system is the block-Jacobi preconditioned reduced S
  const bool eo = (p->flags & COARSE_ODD_EVEN) != 0;
  if (eo)
    for (int i = 0; i < nops; ++i)
      if (!ops[i]->eo_sites) {
        set_error("coarse_solve_batched: COARSE_ODD_EVEN needs even lattice extents (operator %d)", i);
        return COARSE_ERR_INVALID_ARG;
      }

  // ---- setup per operator: polynomial and recycle space through the single-operator solver
  double setup_ms = 0.0;
  bool chain_bf16 = false;
  {
    const double ts = now_ms();
    size_t maxN = 0;
    for (int i = 0; i < nops; ++i) maxN = std::max(maxN, (size_t)ops[i]->V * ops[i]->n);
    double2* tmp = nullptr;
    if (cudaMalloc((void**)&tmp, 2 * maxN * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      set_error("coarse_solve_batched: setup allocation failed");
      return COARSE_ERR_OOM;
    }
    coarse_solve_params ps = *p;
    // COARSE_POLY_BF16: FP32 inner solves whose chain phases read BF16 blocks (every operator
    // must carry them); the setup solves build each recycle space for that same chain
    bool poly_bf16 = (p->flags & COARSE_POLY_BF16) && prec == COARSE_PREC_FP32;
    for (int i = 0; i < nops; ++i) poly_bf16 = poly_bf16 && ops[i]->blk[COARSE_PREC_BF16].ptr != nullptr;
    ps.flags = COARSE_ZERO_GUESS | (poly_bf16 ? COARSE_POLY_BF16 : 0u);
    chain_bf16 = poly_bf16;
    int rc = COARSE_OK;
    for (int i = 0; i < nops && rc == COARSE_OK; ++i) {
      coarse_op* op = ops[i];
      if (!op->blk[prec].ptr) {
        set_error("coarse_solve_batched: precision %d not enabled on operator %d", prec, i);
        rc = COARSE_ERR_INVALID_ARG;
        break;
      }
      Solver* sv = get_solver(op, prec, 0, s, eo ? 1 : 0);
      const int N = op->V * op->n;
      if (eo && (rc = eo_prepare(op, op->mu, s)) != COARSE_OK) break;
      if ((rc = sv->ensure(m, k, d > 0 ? d : 1)) != COARSE_OK) break;
      if (!sv->poly_ok || (d > 0 && sv->d == 0) || (d == 0 && sv->d != 0)) {
        if ((rc = sv->build_poly(nullptr, p->seed + i, d)) != COARSE_OK) break;  // seeded start per operator
      }
      for (int it = 0; k > 0 && sv->updates < p->recycle_updates && it < 3; ++it) {
        if ((rc = launch_fill_gaussian(tmp, N, p->seed * 7919ull + 31ull * i + it, s)) != COARSE_OK) break;
        coarse_solve_info inf;
        // the first setup solve builds the recycle space from a full GMRES(m) cycle (Sec. 3.4)
        coarse_solve_params pi = ps;
        if (sv->k_cur == 0) pi.flags |= COARSE_RECYCLE_FULL_CYCLE;
        int r2 = solve_column(op, sv, tmp, tmp + maxN, &pi, &inf, s, +1);
        if (r2 != COARSE_OK && r2 != COARSE_ERR_NOT_CONVERGED) { rc = r2; break; }
        if (sv->k_cur == 0 && it >= 1) break;  // the solves converge before a recycle space forms
      }
    }
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (rc != COARSE_OK) return rc;
    setup_ms = now_ms() - ts;
  }

  // ---- lockstep batch: descriptors and memory
  Batch B;
  B.prec = prec;
  B.poly_prec = chain_bf16 ? COARSE_PREC_BF16 : prec;
  B.m = m;
  B.dd = d == 0 ? 0 : std::max(d, 2);
  int ns = 0;
  size_t maxN = 0;
  for (int i = 0; i < nops; ++i) {
    ns += nrhs[i];
    maxN = std::max(maxN, (size_t)ops[i]->V * ops[i]->n);
  }
  B.ns = ns;
  B.E = batch_chunk_elems((int)maxN);
  const int maxq = kMaxK + kMaxDense + 2;
  const int ldh = kMaxDense + 1;
  std::vector<size_t> off_vec(ns), off_small(ns);
  std::vector<int> nch(ns), nchf(ns);
  std::vector<int> chunk_off(ns + 1, 0), chunk_off_f(ns + 1, 0);
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t o = bytes; bytes += align256(n); return o; };
  const size_t o_step = take(64);
  const size_t o_states = take(sizeof(CycleState) * ns);
  const size_t o_norms = take(sizeof(double) * 4 * ns);
  const size_t o_flags = take(sizeof(int) * 2 * ns);
  const size_t o_S = take(sizeof(BSolve) * ns);
  const size_t o_coff = take(sizeof(int) * (ns + 1));
  const size_t o_coff_f = take(sizeof(int) * (ns + 1));
  const size_t o_groups = take(sizeof(int) * (2 * ns + 8) * 3);
  const size_t o_egroups = take(sizeof(int) * (2 * ns + 8) * 3);
  const size_t o_ctl = take(sizeof(BCtl));
  const size_t o_info = take(sizeof(BInfo) * ns);
  // multi-RHS stencil phases: BF16 inner solves, every operator carrying the fragment-layout
  // blocks (created with max_nrhs > 1) and at most 12 columns
  B.eo = eo;
  B.mrhs = prec == COARSE_PREC_BF16 && !eo;
  for (int i = 0; i < nops; ++i) B.mrhs = B.mrhs && ops[i]->mrhs.ptr != nullptr && nrhs[i] <= kMrhsColumns;
  std::vector<size_t> off_xb(nops, 0);
  size_t o_mops = 0, o_mgrp = 0, o_woff = 0, o_merr = 0;
  if (B.mrhs) {
    o_mops = take(sizeof(BMOp) * nops);
    size_t groups = 0;
    for (int i = 0; i < nops; ++i) {
      int P, S;
      bm_shape(ops[i]->n, &P, &S);
      groups += (ops[i]->V + P - 1) / P;
    }
    o_mgrp = take(sizeof(int) * ((2 * (size_t)nops + 8) * 3 + groups));
    o_woff = take(sizeof(int) * ((size_t)nops + 1));
    o_merr = take(64);
    for (int i = 0; i < nops; ++i)
      off_xb[i] = take((size_t)ops[i]->V * ((nrhs[i] + 3) / 4) * (ops[i]->n / 16) * 256);
  }
  {
    int sidx = 0;
    for (int i = 0; i < nops; ++i) {
      const int N = ops[i]->V * ops[i]->n;
      const int V = ops[i]->V;
      Solver* sv = eo ? ops[i]->eo_solver[prec] : ops[i]->solver[prec];
      const int kc = sv->k_cur;
      for (int c = 0; c < nrhs[i]; ++c, ++sidx) {
        nch[sidx] = batch_chunks(eo ? N / 2 : N, B.E);
        nchf[sidx] = batch_chunks(N, B.E);
        chunk_off[sidx + 1] = chunk_off[sidx] + nch[sidx];
        chunk_off_f[sidx + 1] = chunk_off_f[sidx] + nchf[sidx];
        off_vec[sidx] = take(sizeof(float2) * (size_t)N * (m + 7) + sizeof(float2) * 5 * (size_t)N +
                             sizeof(double2) * 6 * (size_t)N + sizeof(int) * (V + 4) + 1024);
        off_small[sidx] = take(sizeof(double2) * (2 * (size_t)ldh * kMaxDense + 3 * kMaxDense + (size_t)kMaxK * kMaxDense +
                                                  4 * maxq + 3 * kMaxPoly + 4) +
                               sizeof(double) * 2 * (size_t)kBatchMaxQ * nchf[sidx] + sizeof(void*) * (3 * (kc + m + 2)) +
                               4096);
      }
    }
  }
  B.total_chunks = chunk_off[ns];
  B.total_chunks_f = chunk_off_f[ns];
  if (cudaMalloc((void**)&B.mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("coarse_solve_batched: allocation of %zu bytes failed", bytes);
    return COARSE_ERR_OOM;
  }
  COARSE_CUDA(cudaMemsetAsync(B.mem, 0, bytes, s));
  B.step = reinterpret_cast<int*>(B.mem + o_step);
  B.states = reinterpret_cast<CycleState*>(B.mem + o_states);
  B.norms = reinterpret_cast<double*>(B.mem + o_norms);
  B.flags = reinterpret_cast<int*>(B.mem + o_flags);
  B.dS = reinterpret_cast<BSolve*>(B.mem + o_S);
  B.chunk_off = reinterpret_cast<int*>(B.mem + o_coff);
  B.chunk_off_f = reinterpret_cast<int*>(B.mem + o_coff_f);
  {
    const double2 cst[2] = {make_double2(-1.0, 0.0), make_double2(1.0, 0.0)};
    COARSE_CUDA(cudaMemcpyAsync(B.step + 4, cst, sizeof(cst), cudaMemcpyHostToDevice, s));
    COARSE_CUDA(cudaMemcpyAsync(B.chunk_off, chunk_off.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, s));
    COARSE_CUDA(cudaMemcpyAsync(B.chunk_off_f, chunk_off_f.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, s));
  }
  std::vector<BSolve> hs(ns);
  std::vector<std::vector<void*>> tabs(ns);
  std::vector<std::vector<double2>> polys(ns);
  {
    int sidx = 0;
    for (int i = 0; i < nops; ++i) {
      coarse_op* op = ops[i];
      Solver* sv = eo ? op->eo_solver[prec] : op->solver[prec];
      const int N = op->V * op->n;
      const int kc = sv->k_cur;
      B.any_kc = B.any_kc || kc > 0;
      // chain coefficients padded to the batch degree (see Batch::precondition)
      std::vector<double2> pc(3 * kMaxPoly + 4, make_double2(0.0, 0.0));
      if (B.dd > 0) {
        const int deff = sv->d;
        auto inv = [](double2 z) {
          const double a = z.x * z.x + z.y * z.y;
          return make_double2(z.x / a, -z.y / a);
        };
        const double2 i1 = inv(sv->theta_host[0]);
        for (int st = 1; st < B.dd; ++st) {
          if (st < deff) {
            pc[3 * (st - 1) + 0] = inv(sv->theta_host[st - 1]);
            pc[3 * (st - 1) + 1] = inv(sv->theta_host[st]);
          } else if (st == 1) {
            pc[0] = i1;  // degree one: acc = x / theta_1
          }
          pc[3 * (st - 1) + 2] = i1;
        }
      }
      for (int c = 0; c < nrhs[i]; ++c, ++sidx) {
        BSolve& S = hs[sidx];
        char* v = B.mem + off_vec[sidx];
        char* sm = B.mem + off_small[sidx];
        const size_t vb = sizeof(float2) * (size_t)N;
        S.blk = op->blk[prec].ptr;
        S.blk_poly = op->blk[B.poly_prec].ptr;
        S.blk64 = op->blk[COARSE_PREC_FP64].ptr;
        S.nb = op->nb;
        S.V = op->V;
        S.n = op->n;
        S.N = eo ? N / 2 : N;
        S.Nf = N;
        S.eo = eo ? 1 : 0;
        S.kc = kc;
        S.mu = op->mu;
        std::vector<void*>& T = tabs[sidx];
        for (int j = 0; j <= m; ++j) T.push_back(v + j * vb);
        S.r = v + (m + 1) * vb;
        S.e = v + (m + 2) * vb;
        S.t = v + (m + 3) * vb;
        S.sa = v + (m + 4) * vb;
        S.sb = v + (m + 5) * vb;
        S.acc = v + (m + 6) * vb;
        S.part = v + (m + 7) * vb;
        S.push = v + (m + 8) * vb;
        if (eo) {
          // the half apply keeps no stencil scratch: its 5 N-vector region holds the odd-even work
          const size_t hb = vb / 2;
          char* w = v + (m + 7) * vb;
          S.f32 = w;
          S.re = w + vb;
          S.ro = w + vb + hb;
          S.to = w + vb + 2 * hb;
          S.eoe = w + vb + 3 * hb;
          S.todd = w + vb + 4 * hb;
          S.inv = op->inv[0][prec].ptr;
          S.inv_poly = op->inv[0][B.poly_prec].ptr;
          S.eo_rec = op->eo_rec;
          S.eo_sites = op->eo_sites;
        }
        char* v64 = v + (m + 12) * vb;
        S.r64 = reinterpret_cast<double2*>(v64);
        S.part64 = v64 + sizeof(double2) * (size_t)N;
        S.cnt = reinterpret_cast<int*>(v64 + sizeof(double2) * 6 * (size_t)N);
        S.b64 = static_cast<const double2*>(b[i]) + (size_t)c * N;
        S.x64 = static_cast<double2*>(x[i]) + (size_t)c * N;
        // small dense state
        size_t o = 0;
        auto sub = [&](size_t n) { char* q = sm + o; o += align256(n); return q; };
        S.dn.H = (double2*)sub(sizeof(double2) * ldh * kMaxDense);
        S.dn.R = (double2*)sub(sizeof(double2) * ldh * kMaxDense);
        S.dn.cs = (double*)sub(sizeof(double) * kMaxDense);
        S.dn.sn = (double2*)sub(sizeof(double2) * kMaxDense);
        S.dn.g = (double2*)sub(sizeof(double2) * (kMaxDense + 1));
        S.dn.B = (double2*)sub(sizeof(double2) * kMaxK * kMaxDense);
        S.dn.ycoef = (double2*)sub(sizeof(double2) * maxq);
        S.dn.z = (double2*)sub(sizeof(double2) * maxq);
        S.dn.coefC = S.dn.coefU = nullptr;
        S.dn.theta = nullptr;
        S.dn.polyc = (double2*)sub(sizeof(double2) * (3 * kMaxPoly + 4));
        S.dn.ldh = ldh;
        S.dn.ldb = kMaxK;
        S.polyc = S.dn.polyc;
        S.h1 = (double2*)sub(sizeof(double2) * maxq);
        S.h2 = (double2*)sub(sizeof(double2) * maxq);
        S.partial = (double*)sub(sizeof(double) * 2 * (size_t)kBatchMaxQ * nch[sidx]);
        void** tvt = (void**)sub(sizeof(void*) * (m + 1));
        void** tqt = (void**)sub(sizeof(void*) * (kc + m + 1));
        void** tut = (void**)sub(sizeof(void*) * (kc + m));
        S.counter = (unsigned*)sub(64);
        S.vt = tvt;
        S.qt = tqt;
        S.ut = tut;
        S.st = B.states + sidx;
        S.norm2 = B.norms + 4 * sidx;
        S.flags = B.flags + 2 * sidx;
        S.nch = nch[sidx];
        S.nchf = nchf[sidx];
        // pointer tables: vt = basis, qt = [C, basis], ut = [U, basis]
        std::vector<void*> hq, hu;
        for (int j = 0; j < kc; ++j) hq.push_back(sv->C[sv->par][j]);
        for (int j = 0; j <= m; ++j) hq.push_back(T[j]);
        for (int j = 0; j < kc; ++j) hu.push_back(sv->U[sv->par][j]);
        for (int j = 0; j < m; ++j) hu.push_back(T[j]);
        COARSE_CUDA(cudaMemcpyAsync(tvt, T.data(), sizeof(void*) * (m + 1), cudaMemcpyHostToDevice, s));
        COARSE_CUDA(cudaMemcpyAsync(tqt, hq.data(), sizeof(void*) * hq.size(), cudaMemcpyHostToDevice, s));
        COARSE_CUDA(cudaMemcpyAsync(tut, hu.data(), sizeof(void*) * hu.size(), cudaMemcpyHostToDevice, s));
        polys[sidx] = pc;
        COARSE_CUDA(cudaMemcpyAsync(S.dn.polyc, polys[sidx].data(), sizeof(double2) * pc.size(),
                                    cudaMemcpyHostToDevice, s));
      }
    }
  }
  COARSE_CUDA(cudaMemcpyAsync(B.dS, hs.data(), sizeof(BSolve) * ns, cudaMemcpyHostToDevice, s));
  std::vector<BMOp> hops;
  std::vector<int> woff, mgroup_tab;
  if (B.mrhs) {
    hops.resize(nops);
    woff.assign(nops + 1, 0);
    int s0 = 0;
    long long words = 0;
    for (int i = 0; i < nops; ++i) {
      BMOp& o = hops[i];
      o.frag = ops[i]->mrhs.ptr;
      o.nb = ops[i]->nb;
      o.xb = B.mem + off_xb[i];
      o.V = ops[i]->V;
      o.n = ops[i]->n;
      o.R = nrhs[i];
      o.T = (nrhs[i] + 3) / 4;
      o.s0 = s0;
      o.mu = (float)ops[i]->mu;
      s0 += nrhs[i];
      words += (long long)o.V * o.T * (o.n / 16) * 64;
      if (words >= (1ll << 31)) {
        set_error("coarse_solve_batched: %lld packed vector words exceed the 32-bit index", words);
        return COARSE_ERR_INVALID_ARG;
      }
      woff[i + 1] = (int)words;
    }
    B.dops = reinterpret_cast<BMOp*>(B.mem + o_mops);
    B.nops = nops;
    B.word_off = reinterpret_cast<int*>(B.mem + o_woff);
    B.total_words = woff[nops];
    B.merr = reinterpret_cast<int*>(B.mem + o_merr);
    COARSE_CUDA(cudaMemcpyAsync(B.dops, hops.data(), sizeof(BMOp) * nops, cudaMemcpyHostToDevice, s));
    COARSE_CUDA(cudaMemcpyAsync(B.word_off, woff.data(), sizeof(int) * (nops + 1), cudaMemcpyHostToDevice, s));
    // n-groups: operator lists and prefix sums of their site groups
    std::vector<std::pair<size_t, size_t>> spans;
    for (int n : {16, 32, 48}) {
      MGroup mg;
      mg.n = n;
      bm_shape(n, &mg.P, &mg.S);
      std::vector<int> idx, off(1, 0);
      for (int i = 0; i < nops; ++i)
        if (hops[i].n == n) {
          idx.push_back(i);
          off.push_back(off.back() + (hops[i].V + mg.P - 1) / mg.P);
        }
      if (idx.empty()) continue;
      const size_t at = mgroup_tab.size();
      mgroup_tab.insert(mgroup_tab.end(), idx.begin(), idx.end());
      mgroup_tab.insert(mgroup_tab.end(), off.begin(), off.end());
      for (size_t k = 0; k < idx.size(); ++k)
        for (int g = off[k]; g < off[k + 1]; ++g) mgroup_tab.push_back((int)k);
      int* base = reinterpret_cast<int*>(B.mem + o_mgrp) + at;
      mg.a.S = B.dS;
      mg.a.ops = B.dops;
      mg.a.idx = base;
      mg.a.grp_off = base + idx.size();
      mg.a.grp_op = base + idx.size() + off.size();
      mg.a.count = (int)idx.size();
      mg.a.total_groups = off.back();
      mg.a.step = B.step;
      mg.a.err = B.merr;
      B.mgroups.push_back(mg);
    }
    COARSE_CUDA(cudaMemcpyAsync(B.mem + o_mgrp, mgroup_tab.data(), sizeof(int) * mgroup_tab.size(),
                                cudaMemcpyHostToDevice, s));
  }
  // n-groups of the stencil phases
  {
    int* g0 = reinterpret_cast<int*>(B.mem + o_groups);
    for (int n : {16, 32, 48}) {
      std::vector<int> idx, off(1, 0);
      for (int q = 0; q < ns; ++q)
        if (hs[q].n == n) {
          idx.push_back(q);
          off.push_back(off.back() + hs[q].V);
        }
      if (idx.empty()) continue;
      Group g;
      g.n = n;
      g.count = (int)idx.size();
      g.total = off.back();
      g.sidx = g0;
      g.site_off = g0 + idx.size();
      COARSE_CUDA(cudaMemcpyAsync(g.sidx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
      COARSE_CUDA(cudaMemcpyAsync(g.site_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
      g0 += idx.size() + off.size();
      B.groups.push_back(g);
    }
  }
  // odd-even: n-groups over the half-site counts (one output parity per half apply)
  if (eo) {
    int* g0 = reinterpret_cast<int*>(B.mem + o_egroups);
    for (int n : {16, 32, 48}) {
      std::vector<int> idx, off(1, 0);
      for (int q = 0; q < ns; ++q)
        if (hs[q].n == n) {
          idx.push_back(q);
          off.push_back(off.back() + hs[q].V / 2);
        }
      if (idx.empty()) continue;
      Group g;
      g.n = n;
      g.count = (int)idx.size();
      g.total = off.back();
      g.sidx = g0;
      g.site_off = g0 + idx.size();
      COARSE_CUDA(cudaMemcpyAsync(g.sidx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
      COARSE_CUDA(cudaMemcpyAsync(g.site_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
      g0 += idx.size() + off.size();
      B.egroups.push_back(g);
    }
  }
  int kmin = m;
  for (int q = 0; q < ns; ++q) kmin = std::min(kmin, hs[q].kc);
  B.steps_max = kmin > 0 ? m - kmin : m;
  COARSE_CUDA(cudaStreamSynchronize(s));

  // ---- the whole lockstep solve as one CUDA graph with device-side control
  BCtl* dctl = reinterpret_cast<BCtl*>(B.mem + o_ctl);
  BInfo* dinfo = reinterpret_cast<BInfo*>(B.mem + o_info);
  cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& q : cs) COARSE_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
  struct StreamsGuard {
    cudaStream_t* q;
    ~StreamsGuard() { for (int i = 0; i < 4; ++i) if (q[i]) cudaStreamDestroy(q[i]); }
  } guard{cs};
  COARSE_CUDA(cudaGraphCreate(&B.graph, 0));
  BCtl hc{};
  hc.max_ir = p->max_ir;
  hc.max_cyc = p->max_restarts;
  hc.steps_max = B.steps_max;
  hc.tol = p->tol;
  hc.inner_tol = p->inner_tol;
  COARSE_CUDA(cudaGraphConditionalHandleCreate(&hc.h_ir, B.graph, 0, 0));
  COARSE_CUDA(cudaGraphConditionalHandleCreate(&hc.h_cyc, B.graph, 0, 0));
  COARSE_CUDA(cudaGraphConditionalHandleCreate(&hc.h_step, B.graph, 0, 0));
  COARSE_CUDA(cudaMemcpyAsync(dctl, &hc, sizeof(BCtl), cudaMemcpyHostToDevice, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  cudaGraph_t body_ir = nullptr, body_cyc = nullptr, body_step = nullptr;
  const bool zero_guess = (p->flags & COARSE_ZERO_GUESS) != 0;
  auto step_body = [&](cudaStream_t q) -> int {
    TRY(B.step_sequence(q));
    kb_step_gate<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, B.step, ns, 1);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    return COARSE_OK;
  };
  auto cycle_body = [&](cudaStream_t q) -> int {
    if (B.any_kc) {
      TRY(B.vec(BV_PROJ_DOT, q));
      TRY(B.vec(BV_PROJ_UPD, q));
      TRY(B.elem(BE_COMBINE_U, q));
      int src = BS_T;
      TRY(B.precondition(BS_T, BG_ACTIVE, q, &src));
      TRY(B.elem(BE_AXPY_E_PROJ, q, src, BG_ACTIVE));
    }
    TRY(B.vec(BV_NORM_R, q));
    COARSE_CUDA(cudaMemsetAsync(B.step, 0, sizeof(int), q));
    TRY(launch_bcycle_init(B.dS, ns, m, 0.0, q));
    TRY(B.elem(BE_START, q, BS_ACC, BG_STEP));
    kb_step_gate<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, B.step, ns, 0);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    TRY(add_while(q, hc.h_step, &body_step));
    TRY(capture_body(body_step, cs[3], step_body));
    TRY(launch_bcycle_solve(B.dS, ns, q));
    TRY(B.elem(BE_COMBINE_T, q));
    int src = BS_T;
    TRY(B.precondition(BS_T, BG_TAIL, q, &src));
    TRY(B.elem(BE_AXPY_E, q, src, BG_TAIL));
    TRY(B.vec(BV_RES_UPD, q));
    kb_cycle_end<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, dinfo, ns);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    return COARSE_OK;
  };
  auto ir_body = [&](cudaStream_t q) -> int {
    kb_ir_begin<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, dinfo, ns);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    if (eo) TRY(B.eo_rhs(q));
    else TRY(B.elem(BE_TO_LOW, q));
    TRY(add_while(q, hc.h_cyc, &body_cyc));
    TRY(capture_body(body_cyc, cs[2], cycle_body));
    if (eo) TRY(B.eo_correction(q));
    else TRY(B.elem(BE_ADD_LOW, q));
    TRY(B.residual64(q));
    kb_ir_end<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, dinfo, ns);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    return COARSE_OK;
  };
  auto top = [&](cudaStream_t q) -> int {
    if (zero_guess) TRY(B.elem(BE_ZERO_X, q));
    TRY(B.residual64(q));
    TRY(B.norms64(2, q));
    kb_ctl_start<<<1, kCtlThreads, 0, q>>>(dctl, B.dS, dinfo, ns);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
    TRY(add_while(q, hc.h_ir, &body_ir));
    return capture_body(body_ir, cs[1], ir_body);
  };
  const long long l_build0 = launches_so_far();
  {
    COARSE_CUDA(cudaStreamBeginCaptureToGraph(cs[0], B.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = top(cs[0]);
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs[0], &out);
    if (rc == COARSE_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture (batched solve)");
    if (rc != COARSE_OK) return rc;
    e = cudaGraphInstantiate(&B.gexec, B.graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batched solve)");
  }
  // the capture counted every kernel once; the graph's own accounting follows the replay below
  note_launches(-(launches_so_far() - l_build0));
  COARSE_CUDA(cudaGraphLaunch(B.gexec, s));
  std::vector<BInfo> hinfo(ns);
  BCtl ctl_h{};
  COARSE_CUDA(cudaMemcpyAsync(hinfo.data(), dinfo, sizeof(BInfo) * ns, cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaMemcpyAsync(&ctl_h, dctl, sizeof(BCtl), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  B.launches = (long long)graph_kernels(B.graph) + (long long)ctl_h.ir * (long long)graph_kernels(body_ir) +
               (long long)ctl_h.cycles_run * (long long)graph_kernels(body_cyc) +
               (long long)ctl_h.steps_run * (long long)graph_kernels(body_step);
  std::vector<coarse_solve_info> inf(ns);
  std::vector<double> bn(ns), rn(ns);
  bool any_nonfinite = false;
  for (int q = 0; q < ns; ++q) {
    inf[q].status = hinfo[q].status;
    inf[q].iterations = hinfo[q].iterations;
    inf[q].cycles = hinfo[q].cycles;
    inf[q].ir_steps = hinfo[q].ir_steps;
    bn[q] = hinfo[q].bn;
    rn[q] = hinfo[q].rn;
    any_nonfinite = any_nonfinite || hinfo[q].status == COARSE_ERR_NONFINITE;
  }
  COARSE_CUDA(cudaStreamSynchronize(s));
  const double total_ms = now_ms() - t0;
  const long long launches = launches_so_far() - launches0 + B.launches;
  int worst = COARSE_OK;
  for (int q = 0; q < ns; ++q) {
    inf[q].rel_residual = bn[q] > 0.0 ? rn[q] / bn[q] : 0.0;
    if (inf[q].status == COARSE_OK && inf[q].rel_residual > p->tol) inf[q].status = COARSE_ERR_NOT_CONVERGED;
    inf[q].setup_ms = setup_ms;
    inf[q].solve_ms = total_ms;
    inf[q].kernel_launches = (int)std::min<long long>(launches, 2147483647LL);
    if (inf[q].status == COARSE_ERR_NONFINITE) worst = COARSE_ERR_NONFINITE;
    else if (inf[q].status != COARSE_OK && worst == COARSE_OK) worst = inf[q].status;
  }
  {
    int q = 0;
    for (int i = 0; i < nops; ++i) {
      Solver* sv = eo ? ops[i]->eo_solver[prec] : ops[i]->solver[prec];
      for (int c = 0; c < nrhs[i]; ++c, ++q) inf[q].recycle_updates = sv->updates;
    }
  }
  if (infos) memcpy(infos, inf.data(), sizeof(coarse_solve_info) * ns);
  for (int i = 0; i < nops; ++i) TRY(take_stencil_flag(ops[i], s));
  if (B.mrhs) {
    int h = 0;
    COARSE_CUDA(cudaMemcpy(&h, B.merr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
      set_error("coarse_solve_batched: a bounded wait of the multi-RHS stencil ran out; results are invalid");
      return COARSE_ERR_TIMEOUT;
    }
  }
  if (worst == COARSE_ERR_NOT_CONVERGED) set_error("coarse_solve_batched: some solves missed the tolerance");
  if (worst == COARSE_ERR_NONFINITE) set_error("coarse_solve_batched: non-finite values in some solves");
  (void)any_nonfinite;
  return worst;
}
