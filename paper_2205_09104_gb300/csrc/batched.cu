// coarse_solve_batched: many independent solves of uneven operators advanced in lockstep.
//
// Every (operator, right-hand-side column) is one solve.  Setup (polynomial and the first
// u recycle-space updates) runs per operator through the single-operator solver; the solves
// then share their operator's blocks, polynomial and frozen U_k, C_k.  In the lockstep phase
// each Krylov phase is ONE kernel launch over all solves (per n-group for the stencil), the
// launch sequence of one Arnoldi step is captured once in a CUDA graph and replayed for
// every step (the kernels read the step index from a device counter), and per-solve stop /
// active / done flags on the device skip the solves that are finished.  The host reads one
// array of cycle states per cycle and one array of norms per refinement step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "mrhs_core.cuh"
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
  CycleState* states_h = nullptr;
  double* norms = nullptr;
  double* norms_h = nullptr;
  int* flags = nullptr;
  int* flags_h = nullptr;
  int* chunk_off = nullptr;
  std::vector<Group> groups;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  long long launches = 0;

  ~Batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (mem) cudaFree(mem);
    if (states_h) cudaFreeHost(states_h);
  }

  // one stencil phase over all n-groups (chain: a polynomial-chain phase, on the chain's blocks)
  int apply_phase(int mode, int xsel, int ysel, int coef_off, int gate, cudaStream_t s, bool chain = false) {
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
    return launch_belem(op, dS, ns, chunk_off, total_chunks, E, step, aux, gate, s);
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
    return launch_bnorms64(dS, ns, chunk_off, total_chunks, E, 1, s);
  }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

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
      Solver* sv = get_solver(op, prec, 0, s);
      const int N = op->V * op->n;
      if ((rc = sv->ensure(m, k, d > 0 ? d : 1)) != COARSE_OK) break;
      if (!sv->poly_ok || (d > 0 && sv->d == 0) || (d == 0 && sv->d != 0)) {
        if ((rc = sv->build_poly(nullptr, p->seed + i, d)) != COARSE_OK) break;  // seeded start per operator
      }
      for (int it = 0; k > 0 && sv->updates < p->recycle_updates && it < 3; ++it) {
        if ((rc = launch_fill_gaussian(tmp, N, p->seed * 7919ull + 31ull * i + it, s)) != COARSE_OK) break;
        coarse_solve_info inf;
        int r2 = solve_column(op, sv, tmp, tmp + maxN, &ps, &inf, s, +1);
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
  std::vector<int> nch(ns);
  std::vector<int> chunk_off(ns + 1, 0);
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t o = bytes; bytes += align256(n); return o; };
  const size_t o_step = take(64);
  const size_t o_states = take(sizeof(CycleState) * ns);
  const size_t o_norms = take(sizeof(double) * 4 * ns);
  const size_t o_flags = take(sizeof(int) * 2 * ns);
  const size_t o_S = take(sizeof(BSolve) * ns);
  const size_t o_coff = take(sizeof(int) * (ns + 1));
  const size_t o_groups = take(sizeof(int) * (2 * ns + 8) * 3);
  // multi-RHS stencil phases: BF16 inner solves, every operator carrying the fragment-layout
  // blocks (created with max_nrhs > 1) and at most 12 columns
  B.mrhs = prec == COARSE_PREC_BF16;
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
      Solver* sv = ops[i]->solver[prec];
      const int kc = sv->k_cur;
      for (int c = 0; c < nrhs[i]; ++c, ++sidx) {
        nch[sidx] = batch_chunks(N, B.E);
        chunk_off[sidx + 1] = chunk_off[sidx] + nch[sidx];
        off_vec[sidx] = take(sizeof(float2) * (size_t)N * (m + 7) + sizeof(float2) * 5 * (size_t)N +
                             sizeof(double2) * 6 * (size_t)N + sizeof(int) * (V + 4) + 1024);
        off_small[sidx] = take(sizeof(double2) * (2 * (size_t)ldh * kMaxDense + 3 * kMaxDense + (size_t)kMaxK * kMaxDense +
                                                  4 * maxq + 3 * kMaxPoly + 4) +
                               sizeof(double) * 2 * (size_t)kBatchMaxQ * nch[sidx] + sizeof(void*) * (3 * (kc + m + 2)) +
                               4096);
      }
    }
  }
  B.total_chunks = chunk_off[ns];
  if (cudaMalloc((void**)&B.mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("coarse_solve_batched: allocation of %zu bytes failed", bytes);
    return COARSE_ERR_OOM;
  }
  COARSE_CUDA(cudaMemsetAsync(B.mem, 0, bytes, s));
  COARSE_CUDA(cudaMallocHost((void**)&B.states_h, sizeof(CycleState) * ns + sizeof(double) * 4 * ns + sizeof(int) * 2 * ns + 64));
  B.norms_h = reinterpret_cast<double*>(B.states_h + ns);
  B.flags_h = reinterpret_cast<int*>(B.norms_h + 4 * ns);
  B.step = reinterpret_cast<int*>(B.mem + o_step);
  B.states = reinterpret_cast<CycleState*>(B.mem + o_states);
  B.norms = reinterpret_cast<double*>(B.mem + o_norms);
  B.flags = reinterpret_cast<int*>(B.mem + o_flags);
  B.dS = reinterpret_cast<BSolve*>(B.mem + o_S);
  B.chunk_off = reinterpret_cast<int*>(B.mem + o_coff);
  {
    const double2 cst[2] = {make_double2(-1.0, 0.0), make_double2(1.0, 0.0)};
    COARSE_CUDA(cudaMemcpyAsync(B.step + 4, cst, sizeof(cst), cudaMemcpyHostToDevice, s));
    COARSE_CUDA(cudaMemcpyAsync(B.chunk_off, chunk_off.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, s));
  }
  std::vector<BSolve> hs(ns);
  std::vector<std::vector<void*>> tabs(ns);
  std::vector<std::vector<double2>> polys(ns);
  {
    int sidx = 0;
    for (int i = 0; i < nops; ++i) {
      coarse_op* op = ops[i];
      Solver* sv = op->solver[prec];
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
        S.N = N;
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
  int kmin = m;
  for (int q = 0; q < ns; ++q) kmin = std::min(kmin, hs[q].kc);
  B.steps_max = kmin > 0 ? m - kmin : m;
  COARSE_CUDA(cudaEventCreateWithFlags(&B.ev[0], cudaEventDisableTiming));
  COARSE_CUDA(cudaEventCreateWithFlags(&B.ev[1], cudaEventDisableTiming));
  COARSE_CUDA(cudaStreamSynchronize(s));

  // ---- the Arnoldi step as a CUDA graph
  {
    cudaStream_t cs;
    COARSE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? B.step_sequence(cs) : cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t e2 = cudaStreamEndCapture(cs, &B.graph);
    if (rc == COARSE_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
    if (rc == COARSE_OK) {
      e2 = cudaGraphInstantiate(&B.gexec, B.graph, 0);
      if (e2 != cudaSuccess) rc = cuda_fail(e2, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cs);
    if (rc != COARSE_OK) return rc;
  }
  size_t graph_nodes = 0;
  cudaGraphGetNodes(B.graph, nullptr, &graph_nodes);

  // ---- lockstep refinement
  std::vector<coarse_solve_info> inf(ns);
  std::vector<double> bn(ns), rn(ns);
  std::vector<int> done(ns, 0), active(ns, 0);
  auto put_flags = [&]() -> int {
    for (int q = 0; q < ns; ++q) {
      B.flags_h[2 * q] = active[q];
      B.flags_h[2 * q + 1] = done[q];
    }
    COARSE_CUDA(cudaMemcpyAsync(B.flags, B.flags_h, sizeof(int) * 2 * ns, cudaMemcpyHostToDevice, s));
    return COARSE_OK;
  };
  auto get_norms = [&]() -> int {
    COARSE_CUDA(cudaMemcpyAsync(B.norms_h, B.norms, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost, s));
    COARSE_CUDA(cudaStreamSynchronize(s));
    return COARSE_OK;
  };
  TRY(put_flags());
  if (p->flags & COARSE_ZERO_GUESS) TRY(B.elem(BE_ZERO_X, s));
  TRY(B.residual64(s));
  TRY(launch_bnorms64(B.dS, ns, B.chunk_off, B.total_chunks, B.E, 2, s));
  TRY(get_norms());
  bool any_nonfinite = false;
  for (int q = 0; q < ns; ++q) {
    bn[q] = sqrt(B.norms_h[4 * q + 2]);
    rn[q] = sqrt(B.norms_h[4 * q + 1]);
    if (!isfinite(bn[q]) || !isfinite(rn[q])) {
      inf[q].status = COARSE_ERR_NONFINITE;
      done[q] = 1;
      any_nonfinite = true;
    } else {
      done[q] = (bn[q] == 0.0 || rn[q] <= p->tol * bn[q]) ? 1 : 0;
    }
  }
  for (int ir = 0; ir < p->max_ir; ++ir) {
    int left = 0;
    for (int q = 0; q < ns; ++q) left += !done[q];
    if (left == 0) break;
    for (int q = 0; q < ns; ++q) {
      active[q] = !done[q];
      B.norms_h[4 * q + 3] = std::max(p->inner_tol, 0.5 * p->tol * bn[q] / std::max(rn[q], 1e-300));
    }
    COARSE_CUDA(cudaMemcpyAsync(B.norms, B.norms_h, sizeof(double) * 4 * ns, cudaMemcpyHostToDevice, s));
    TRY(put_flags());
    TRY(B.elem(BE_TO_LOW, s));
    for (int cyc = 0; cyc < p->max_restarts; ++cyc) {
      int act = 0;
      for (int q = 0; q < ns; ++q) act += active[q];
      if (act == 0) break;
      if (B.any_kc) {
        TRY(B.vec(BV_PROJ_DOT, s));
        TRY(B.vec(BV_PROJ_UPD, s));
        TRY(B.elem(BE_COMBINE_U, s));
        int src = BS_T;
        TRY(B.precondition(BS_T, BG_ACTIVE, s, &src));
        TRY(B.elem(BE_AXPY_E_PROJ, s, src, BG_ACTIVE));
      }
      TRY(B.vec(BV_NORM_R, s));
      COARSE_CUDA(cudaMemsetAsync(B.step, 0, sizeof(int), s));
      TRY(launch_bcycle_init(B.dS, ns, m, 0.0, s));
      TRY(B.elem(BE_START, s, BS_ACC, BG_STEP));
      // steps: graph replays in chunks of 4, stop flags read back one chunk behind
      int pending = -1;
      for (int j0 = 0; j0 < B.steps_max; j0 += 4) {
        for (int j = j0; j < B.steps_max && j < j0 + 4; ++j) {
          COARSE_CUDA(cudaGraphLaunch(B.gexec, s));
          B.launches += (long long)graph_nodes;
        }
        const int slot = (j0 / 4) & 1;
        COARSE_CUDA(cudaMemcpyAsync(B.states_h, B.states, sizeof(CycleState) * ns, cudaMemcpyDeviceToHost, s));
        COARSE_CUDA(cudaEventRecord(B.ev[slot], s));
        if (pending >= 0) {
          COARSE_CUDA(cudaEventSynchronize(B.ev[pending]));
          bool all = true;
          for (int q = 0; q < ns && all; ++q) all = B.states_h[q].stop != 0;
          if (all) break;
        }
        pending = slot;
      }
      COARSE_CUDA(cudaMemcpyAsync(B.states_h, B.states, sizeof(CycleState) * ns, cudaMemcpyDeviceToHost, s));
      COARSE_CUDA(cudaStreamSynchronize(s));
      std::vector<CycleState> cs(B.states_h, B.states_h + ns);
      TRY(launch_bcycle_solve(B.dS, ns, s));
      TRY(B.elem(BE_COMBINE_T, s));
      int src = BS_T;
      TRY(B.precondition(BS_T, BG_TAIL, s, &src));
      TRY(B.elem(BE_AXPY_E, s, src, BG_TAIL));
      TRY(B.vec(BV_RES_UPD, s));
      for (int q = 0; q < ns; ++q) {
        if (!active[q]) continue;
        inf[q].cycles++;
        inf[q].iterations += cs[q].j;
        if (cs[q].status & ST_NONFINITE) {
          inf[q].status = COARSE_ERR_NONFINITE;
          done[q] = 1;
          active[q] = 0;
          any_nonfinite = true;
          continue;
        }
        if (cs[q].j == 0 || cs[q].resid <= cs[q].target || (cs[q].status & (ST_LUCKY | ST_ZERO))) active[q] = 0;
      }
      TRY(put_flags());
    }
    TRY(B.elem(BE_ADD_LOW, s));
    TRY(B.residual64(s));
    TRY(get_norms());
    for (int q = 0; q < ns; ++q) {
      if (done[q]) continue;
      inf[q].ir_steps++;
      rn[q] = sqrt(B.norms_h[4 * q + 1]);
      if (!isfinite(rn[q])) {
        inf[q].status = COARSE_ERR_NONFINITE;
        done[q] = 1;
        any_nonfinite = true;
      } else if (rn[q] <= p->tol * bn[q]) {
        done[q] = 1;
      }
    }
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
      Solver* sv = ops[i]->solver[prec];
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
