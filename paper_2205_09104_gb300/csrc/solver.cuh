// Per-operator, per-precision Krylov solver state (host object owning device memory).
#pragma once

#include <map>

#include <vector>

#include "common.cuh"
#include "solver_state.cuh"

namespace coarse {

struct InnerInfo {
  int cycles = 0;
  int iterations = 0;
  int recycle_failures = 0;
  int breakdowns = 0;  // pipelined cycles ended by t < 0 (Sec. 3.5)
  double last_resid = 0.0;
};

struct Solver {
  coarse_op* op = nullptr;
  int prec = COARSE_PREC_FP32;  // block precision
  int v64 = 0;                  // vectors are complex128
  int N = 0;                    // unknowns
  double mu_eff = 0.0;          // twisted mass entering the apply (sign flipped for the adjoint system)
  cudaStream_t stream = nullptr;
  void* tmp64 = nullptr;        // FP64 work vector owned by the operator

  int m_cap = 0, k_cap = 0, d_cap = 0;
  void* vecmem = nullptr;
  void* smallmem = nullptr;
  std::vector<void*> V;
  std::vector<void*> U[2], C[2];
  int par = 0;       // current U/C buffer
  int k_cur = 0;     // recycle vectors held
  int updates = 0;   // recycle-space updates made
  void *r = nullptr, *e = nullptr, *t = nullptr, *sa = nullptr, *sb = nullptr, *acc = nullptr, *w = nullptr,
       *tmp = nullptr;
  void** vtab = nullptr;
  void** qtab[2] = {nullptr, nullptr};
  void** utab[2] = {nullptr, nullptr};
  void** cnew[2] = {nullptr, nullptr};
  void** unew[2] = {nullptr, nullptr};
  void** one_acc = nullptr;
  void** one_t = nullptr;
  double2 *h1 = nullptr, *h2 = nullptr, *SW = nullptr;
  int ldsw = 0;
  Dense dn{};
  double* partial = nullptr;
  unsigned* counter = nullptr;
  double* norm2 = nullptr;
  CycleState* st = nullptr;
  CycleState* st_host = nullptr;
  int* stop_host = nullptr;             // pinned: stop flags of the last two step chunks
  cudaEvent_t chunk_ev[2] = {nullptr, nullptr};

  int d = 0;             // polynomial degree in use
  bool poly_ok = false;  // polynomial built for the current operator values
  std::vector<double2> theta_host;
  double2 theta1_inv{0.0, 0.0};
  long long matvecs = 0;
  // optional CUDA-event timing of the stencil launches (COARSE_TIME_APPLY)
  bool time_apply = false;
  int cur_tag = -1;                 // Arnoldi step of the applies being launched (-1: not gated)
  struct Timed { int tag; cudaEvent_t a, b; double bytes; bool graph_owned = false; int bprec = 0; };
  std::vector<Timed> timed;         // launched, not yet harvested
  std::vector<cudaEvent_t> ev_pool;
  double apply_ms = 0.0;
  double apply_bytes = 0.0;         // algorithmic bytes of the timed launches
  long long apply_count = 0;
  double prec_ms[3] = {0.0, 0.0, 0.0};      // the same, split by the block precision of the launch
  double prec_bytes[3] = {0.0, 0.0, 0.0};
  long long prec_count[3] = {0, 0, 0};
  // blocks of the polynomial-chain applies (COARSE_POLY_BF16: BF16 while the Krylov operator keeps
  // `prec`); the recycle space belongs to the preconditioned operator of `rec_poly_prec`
  // COARSE_RECYCLE_FULL_CYCLE: while no recycle space is held, cycles run all their steps
  bool full_first = false;
  // COARSE_PIPELINED (Sec. 3.5): latency-1 pipelined Arnoldi.  Va[i] = A V[i] alongside the basis,
  // VC[p][j] = A C[p][j] for the recycle vectors; the reduction of a step runs on aux_stream while
  // the stencil of the same step runs on `stream`.
  bool pipelined = false;
  bool p1_active = false;                // the current cycle is a pipelined one
  bool p1_off = false;                   // this solve fell back to classical cycles
  void* p1mem = nullptr;
  std::vector<void*> Va;
  std::vector<void*> VC[2];
  void** vatab = nullptr;                // [Va_0..Va_m]
  void** atab[2] = {nullptr, nullptr};   // [VC[p], Va_0..Va_m]
  int vc_par = -1, vc_updates = -1, vc_k = -1, vc_poly = -1;   // what VC was computed for
  int poly_builds = 0;
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void** tabs_base = nullptr;
  size_t tabs_used = 0, tabs_cap = 0;
  int ensure_p1();
  int ensure_vc(int kc);
  int p1_step(int j, int kc, void* const* tab);
  int poly_prec = COARSE_PREC_FP32;
  int rec_poly_prec = -1;
  // odd-even: the Krylov operator is S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe on the even sites
  // (N = V n / 2); eo_t is the odd-site scratch of its half applies
  int eo = 0;
  void* eo_t = nullptr;
  // Arnoldi-step chunks captured as CUDA graphs (after the solver's first eager cycle, so that
  // every autotuner decision is made), replayed for every later cycle with the same shape
  struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;           // kernels in the graph (launch accounting on replay)
    long long matvecs = 0;           // operator applies in the graph
    std::vector<Timed> timed_tpl;    // timing events recorded by the graph's event nodes
  };
  std::map<unsigned long long, ChunkGraph> graphs;
  int cycles_done = 0;
  cudaStream_t cap_stream = nullptr;
  void clear_graphs();
  int run_chunk(int j0, int cnt, int kc, void* const* tab);
  void harvest(int steps_done);     // after a stream sync: add the elapsed time of the applies that ran

  ~Solver();
  void release();
  int ensure(int m, int k, int dmax);
  int apply(const void* x, void* y, int mode, void* accp, const double2* coef, const int* stop, int bprec = -1);
  int precondition(const void* v, const void** res, const int* stop);
  int opA(const void* v, void* out, const int* stop);
  int read_state();
  int arnoldi_step(int j, int kc, void* const* tab);
  int build_poly(const double2* start64, uint64_t seed, int d);
  int inner(double target_abs, int max_cycles, int m, int kdef, int ulimit, InnerInfo* info);
  // defects of the held recycle space: out[0] = max_i ||A u_i - c_i|| / ||c_i||,
  // out[1] = max_ij |(C^H C - I)_ij|, out[2] = k held, out[3] = updates made (synchronises stream)
  int recycle_check(double out[4]);
  void invalidate() {
    clear_graphs();
    vc_par = vc_updates = vc_k = vc_poly = -1;
    poly_ok = false;
    d = 0;
    k_cur = 0;
    updates = 0;
    par = 0;
  }
};

// One right-hand side through FP64 iterative refinement around Solver::inner.
// b64, x64: device complex128 [V][n].  mu_sign = +1 (D_c) or -1 (D_c(-mu), adjoint systems).
int solve_column(coarse_op* op, Solver* s, const double2* b64, double2* x64, const coarse_solve_params* p,
                 coarse_solve_info* info, cudaStream_t stream, int mu_sign);

Solver* get_solver(coarse_op* op, int prec, int adjoint_system, cudaStream_t stream, int odd_even = 0);

}  // namespace coarse
