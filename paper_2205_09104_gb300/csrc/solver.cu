// Host side of the coarsest-level solver (Sec. 3.6): the launch sequence of
// restarted GMRES / GCRO-DR with the polynomial right preconditioner, inside
// FP64 iterative refinement.  Every vector and small dense operation runs in
// the library's kernels; the host reads back one small status record per
// Arnoldi cycle (and per refinement step) to decide what to launch next.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "common.cuh"
#include "oddeven.cuh"
#include "solver.cuh"
#include "solver_state.cuh"

namespace coarse {

namespace {

size_t csize(int v64) { return v64 ? sizeof(double2) : sizeof(float2); }

template <class T>
int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
    return COARSE_ERR_OOM;
  }
  return COARSE_OK;
}

#define TRY(call)                 \
  do {                            \
    int _rc = (call);             \
    if (_rc != COARSE_OK) return _rc; \
  } while (0)

}  // namespace

Solver::~Solver() { release(); }

void Solver::clear_graphs() {
  for (auto& kv : graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (const Timed& tm : kv.second.timed_tpl) {
      ev_pool.push_back(tm.a);
      ev_pool.push_back(tm.b);
    }
  }
  graphs.clear();
  // replayed entries of graph-owned events may still sit in `timed`: their events went back above
  std::vector<Timed> keep;
  for (const Timed& tm : timed)
    if (!tm.graph_owned) keep.push_back(tm);
  timed.swap(keep);
  cycles_done = 0;
}

// Steps j0 .. j0+cnt-1 of the current cycle: eager launches for the solver's first cycle and
// for solves that time their stencil launches (COARSE_TIME_APPLY: per-launch events), otherwise a
// CUDA graph per (j0, cnt, kc, recycle parity, chain precision, degree) captured once, replayed.
int Solver::run_chunk(int j0, int cnt, int kc, void* const* tab) {
  auto issue = [&]() -> int {
    for (int j = j0; j < j0 + cnt; ++j) {
      cur_tag = j;
      if (p1_active) {
        TRY(p1_step(j, kc, tab));
      } else {
        TRY(opA(V[j], V[j + 1], &st->stop));
        TRY(arnoldi_step(j, kc, tab));
      }
    }
    return COARSE_OK;
  };
  if (cycles_done < 1 || time_apply) return issue();
  const unsigned long long key = (unsigned long long)j0 | ((unsigned long long)cnt << 8) |
                                 ((unsigned long long)kc << 16) | ((unsigned long long)par << 24) |
                                 ((unsigned long long)poly_prec << 26) | ((unsigned long long)d << 28) |
                                 ((unsigned long long)(p1_active ? 1 : 0) << 36);
  auto it = graphs.find(key);
  if (it == graphs.end()) {
    if (!cap_stream) COARSE_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    ChunkGraph g;
    const cudaStream_t user = stream;
    const long long l0 = launches_so_far(), mv0 = matvecs;
    const size_t t0 = timed.size();
    stream = cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? issue() : cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t e2 = cudaStreamEndCapture(cap_stream, &graph);
    stream = user;
    if (rc == COARSE_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
    if (rc == COARSE_OK) {
      e2 = cudaGraphInstantiate(&g.exec, graph, 0);
      if (e2 != cudaSuccess) rc = cuda_fail(e2, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    g.kernels = launches_so_far() - l0;
    g.matvecs = matvecs - mv0;
    g.timed_tpl.assign(timed.begin() + t0, timed.end());
    for (Timed& tm : g.timed_tpl) tm.graph_owned = true;
    timed.resize(t0);
    // the capture counted its launches and applies once: they run only when replayed
    note_launches(-g.kernels);
    matvecs = mv0;
    if (rc != COARSE_OK) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (const Timed& tm : g.timed_tpl) {
        ev_pool.push_back(tm.a);
        ev_pool.push_back(tm.b);
      }
      return rc;
    }
    it = graphs.emplace(key, std::move(g)).first;
  }
  COARSE_CUDA(cudaGraphLaunch(it->second.exec, stream));
  note_launches(it->second.kernels);
  matvecs += it->second.matvecs;
  for (const Timed& tm : it->second.timed_tpl) timed.push_back(tm);
  return COARSE_OK;
}

void Solver::release() {
  clear_graphs();
  if (cap_stream) {
    cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
  }
  for (const Timed& tm : timed) {
    ev_pool.push_back(tm.a);
    ev_pool.push_back(tm.b);
  }
  timed.clear();
  for (cudaEvent_t ev : ev_pool) cudaEventDestroy(ev);
  ev_pool.clear();
  for (int i = 0; i < 2; ++i)
    if (chunk_ev[i]) { cudaEventDestroy(chunk_ev[i]); chunk_ev[i] = nullptr; }
  if (vecmem) cudaFree(vecmem);
  if (smallmem) cudaFree(smallmem);
  if (p1mem) cudaFree(p1mem);
  p1mem = nullptr;
  Va.clear();
  VC[0].clear();
  VC[1].clear();
  vatab = atab[0] = atab[1] = nullptr;
  vc_par = vc_updates = vc_k = vc_poly = -1;
  if (aux_stream) { cudaStreamDestroy(aux_stream); aux_stream = nullptr; }
  if (ev_fork) { cudaEventDestroy(ev_fork); ev_fork = nullptr; }
  if (ev_join) { cudaEventDestroy(ev_join); ev_join = nullptr; }
  if (st_host) cudaFreeHost(st_host);
  vecmem = nullptr;
  smallmem = nullptr;
  st_host = nullptr;
  m_cap = k_cap = d_cap = 0;
  k_cur = 0;
  updates = 0;
  d = 0;
  poly_ok = false;
}

int Solver::ensure(int m, int k, int dmax) {
  if (m <= m_cap && k == k_cap && dmax <= d_cap && vecmem) return COARSE_OK;
  release();
  m_cap = m;
  k_cap = k;
  d_cap = dmax;
  const size_t cs = csize(v64);
  const size_t nvec = (size_t)(m + 1) + 4 * (size_t)k + 9;
  const size_t vbytes = cs * (size_t)N;
  TRY(dalloc((char**)&vecmem, nvec * vbytes));
  char* p = (char*)vecmem;
  auto take = [&]() { void* q = p; p += vbytes; return q; };
  V.assign(m + 1, nullptr);
  for (int i = 0; i <= m; ++i) V[i] = take();
  for (int b = 0; b < 2; ++b) {
    U[b].assign(k, nullptr);
    C[b].assign(k, nullptr);
    for (int i = 0; i < k; ++i) U[b][i] = take();
    for (int i = 0; i < k; ++i) C[b][i] = take();
  }
  r = take(); e = take(); t = take(); sa = take(); sb = take(); acc = take(); w = take(); tmp = take();
  eo_t = take();
  // small arrays
  const int ldh = kMaxDense + 1;
  const int maxq = kMaxK + kMaxDense + 2;
  ldsw = maxq;
  size_t nsmall = 0;
  auto cnt = [&](size_t c) { size_t o = nsmall; nsmall += (c * sizeof(double2) + 255) / 256 * 256; return o; };
  const size_t o_h1 = cnt(maxq), o_h2 = cnt(maxq), o_H = cnt((size_t)ldh * kMaxDense), o_R = cnt((size_t)ldh * kMaxDense);
  const size_t o_cs = cnt(kMaxDense), o_sn = cnt(kMaxDense), o_g = cnt(kMaxDense + 1), o_B = cnt((size_t)kMaxK * kMaxDense);
  const size_t o_y = cnt(maxq), o_z = cnt(maxq), o_cC = cnt((size_t)maxq * kMaxK), o_cU = cnt((size_t)maxq * kMaxK);
  const size_t o_th = cnt(kMaxPoly + 1), o_pc = cnt(kPolyScale + 1), o_SW = cnt((size_t)kMaxK * maxq);
  const int nch = max_reduction_chunks(N) > 304 ? max_reduction_chunks(N) : 304;
  const size_t o_part = cnt((size_t)(maxq + 8) * nch), o_st = cnt(sizeof(CycleState) / sizeof(double2) + 1);
  const size_t o_n2 = cnt(8), o_cnt = cnt(4), o_tab = cnt(16 * (size_t)(2 * maxq + 8));
  TRY(dalloc((char**)&smallmem, nsmall));
  char* b = (char*)smallmem;
  h1 = (double2*)(b + o_h1); h2 = (double2*)(b + o_h2);
  dn.H = (double2*)(b + o_H); dn.R = (double2*)(b + o_R); dn.cs = (double*)(b + o_cs); dn.sn = (double2*)(b + o_sn);
  dn.g = (double2*)(b + o_g); dn.B = (double2*)(b + o_B); dn.ycoef = (double2*)(b + o_y); dn.z = (double2*)(b + o_z);
  dn.coefC = (double2*)(b + o_cC); dn.coefU = (double2*)(b + o_cU); dn.theta = (double2*)(b + o_th);
  dn.polyc = (double2*)(b + o_pc);
  dn.ldh = ldh;
  dn.ldb = kMaxK > 0 ? kMaxK : 1;
  SW = (double2*)(b + o_SW);
  partial = (double*)(b + o_part);
  st = (CycleState*)(b + o_st);
  norm2 = (double*)(b + o_n2);
  counter = (unsigned*)(b + o_cnt);
  void** tabs = (void**)(b + o_tab);
  COARSE_CUDA(cudaMemsetAsync(smallmem, 0, nsmall, stream));
  // pointer tables: vtab = [V_0..V_m]; qtab[p] = [C[p], V]; utab[p] = [U[p], V]; cnew[p] = C[1-p]; unew[p] = U[1-p]
  std::vector<void*> host;
  auto put = [&](const std::vector<void*>& v) { void** at = tabs + host.size(); host.insert(host.end(), v.begin(), v.end()); return at; };
  vtab = put(V);
  for (int p = 0; p < 2; ++p) {
    std::vector<void*> q(C[p]);
    q.insert(q.end(), V.begin(), V.end());
    qtab[p] = put(q);
    std::vector<void*> u(U[p]);
    u.insert(u.end(), V.begin(), V.end());
    utab[p] = put(u);
    cnew[p] = put(C[1 - p]);
    unew[p] = put(U[1 - p]);
  }
  one_acc = put({acc});
  one_t = put({t});
  COARSE_CUDA(cudaMemcpyAsync(tabs, host.data(), host.size() * sizeof(void*), cudaMemcpyHostToDevice, stream));
  tabs_base = tabs;
  tabs_used = host.size();
  tabs_cap = 16 * (size_t)(2 * maxq + 8) * sizeof(double2) / sizeof(void*);
  COARSE_CUDA(cudaMallocHost((void**)&st_host, sizeof(CycleState) + 4 * sizeof(int)));
  stop_host = (int*)(st_host + 1);
  for (int i = 0; i < 2; ++i)
    if (!chunk_ev[i]) COARSE_CUDA(cudaEventCreateWithFlags(&chunk_ev[i], cudaEventDisableTiming));
  COARSE_CUDA(cudaStreamSynchronize(stream));
  par = 0;
  k_cur = 0;
  updates = 0;
  poly_ok = false;
  d = 0;
  return COARSE_OK;
}

int Solver::apply(const void* x, void* y, int mode, void* accp, const double2* coef, const int* stop, int bprec) {
  if (bprec < 0) bprec = prec;
  auto launch = [&]() -> int {
    if (eo) return launch_eo_schur(op, bprec, mu_eff, x, y, eo_t, mode, accp, coef, stop, stream);
    ApplyArgs a = make_apply_args(op, bprec, x, y);
    a.acc = accp;
    a.coef = coef;
    a.mu = mu_eff;
    a.mode = mode;
    a.stop = stop;
    return launch_apply(bprec, op->n, a, stream);
  };
  ++matvecs;
  if (!time_apply) return launch();
  while (ev_pool.size() < 2) {
    cudaEvent_t ev;
    COARSE_CUDA(cudaEventCreate(&ev));
    ev_pool.push_back(ev);
  }
  // algorithmic bytes: full stencil 5 n^2 V blocks + vector in/out; S: two half applies, each
  // reading 4.5 n^2 V block entries, with vector traffic 2.5 x (V n) (in, out, odd intermediate)
  const double esz[3] = {16.0, 8.0, 4.0}, vsz = v64 ? 16.0 : 8.0;
  const double nn = (double)op->n * op->n * (double)op->V, vn = (double)op->V * op->n;
  const double bytes = eo ? 9.0 * nn * esz[bprec] + 2.5 * vn * vsz : 5.0 * nn * esz[bprec] + 2.0 * (double)N * vsz;
  Timed tm{cur_tag, ev_pool.back(), nullptr, bytes};
  tm.bprec = bprec;
  ev_pool.pop_back();
  tm.b = ev_pool.back();
  ev_pool.pop_back();
  COARSE_CUDA(cudaEventRecord(tm.a, stream));
  TRY(launch());
  COARSE_CUDA(cudaEventRecord(tm.b, stream));
  timed.push_back(tm);
  return COARSE_OK;
}

void Solver::harvest(int steps_done) {
  for (const Timed& tm : timed) {
    if (tm.tag < 0 || tm.tag < steps_done) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, tm.a, tm.b) == cudaSuccess) {
        apply_ms += ms;
        apply_bytes += tm.bytes;
        ++apply_count;
        prec_ms[tm.bprec] += ms;
        prec_bytes[tm.bprec] += tm.bytes;
        ++prec_count[tm.bprec];
      }
    }
    if (!tm.graph_owned) {
      ev_pool.push_back(tm.a);
      ev_pool.push_back(tm.b);
    }
  }
  timed.clear();
}

// out = q(A) v (precondition only, result pointer returned in *res) -- d-1 applies
int Solver::precondition(const void* v, const void** res, const int* stop) {
  if (d == 0) { *res = v; return COARSE_OK; }
  if (d == 1) {  // q = 1/theta_1
    TRY(launch_scale(v64, v, nullptr, theta1_inv, acc, N, stop, 0, stream));
    *res = acc;
    return COARSE_OK;
  }
  TRY(apply(v, sa, APPLY_POLY_FIRST, acc, dn.polyc, stop, poly_prec));
  void* cur = sa;
  void* nxt = sb;
  for (int i = 2; i < d; ++i) {
    TRY(apply(cur, nxt, APPLY_POLY, acc, dn.polyc + 3 * (i - 1), stop, poly_prec));
    void* tt = cur; cur = nxt; nxt = tt;
  }
  *res = acc;
  return COARSE_OK;
}

// out = A v = D q(D) v  (d applies)
int Solver::opA(const void* v, void* out, const int* stop) {
  const void* mv = nullptr;
  TRY(precondition(v, &mv, stop));
  return apply(mv, out, APPLY_PLAIN, nullptr, nullptr, stop);
}

int Solver::read_state() {
  COARSE_CUDA(cudaMemcpyAsync(st_host, st, sizeof(CycleState), cudaMemcpyDeviceToHost, stream));
  COARSE_CUDA(cudaStreamSynchronize(stream));
  return COARSE_OK;
}

// Storage of the pipelined process: Va (m + 1 vectors), VC (2 x k), their pointer tables.
int Solver::ensure_p1() {
  if (p1mem) return COARSE_OK;
  const size_t vbytes = csize(v64) * (size_t)N;
  const size_t nvec = (size_t)(m_cap + 1) + 2 * (size_t)k_cap;
  TRY(dalloc((char**)&p1mem, nvec * vbytes));
  char* p = (char*)p1mem;
  auto take = [&]() { void* q = p; p += vbytes; return q; };
  Va.assign(m_cap + 1, nullptr);
  for (int i = 0; i <= m_cap; ++i) Va[i] = take();
  for (int b = 0; b < 2; ++b) {
    VC[b].assign(k_cap, nullptr);
    for (int i = 0; i < k_cap; ++i) VC[b][i] = take();
  }
  std::vector<void*> host;
  host.insert(host.end(), Va.begin(), Va.end());
  for (int b = 0; b < 2; ++b) {
    host.insert(host.end(), VC[b].begin(), VC[b].end());
    host.insert(host.end(), Va.begin(), Va.end());
  }
  if (tabs_used + host.size() > tabs_cap) {
    set_error("pipelined Arnoldi: pointer table overflow");
    return COARSE_ERR_INVALID_ARG;
  }
  void** at = tabs_base + tabs_used;
  vatab = at;
  atab[0] = at + (m_cap + 1);
  atab[1] = atab[0] + k_cap + (m_cap + 1);
  COARSE_CUDA(cudaMemcpyAsync(at, host.data(), host.size() * sizeof(void*), cudaMemcpyHostToDevice, stream));
  tabs_used += host.size();
  if (!aux_stream) COARSE_CUDA(cudaStreamCreateWithFlags(&aux_stream, cudaStreamNonBlocking));
  if (!ev_fork) COARSE_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  if (!ev_join) COARSE_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  COARSE_CUDA(cudaStreamSynchronize(stream));
  return COARSE_OK;
}

// VC[par][i] = A C[par][i] (Sec. 3.5, the recycle vectors' images under the preconditioned
// operator), recomputed whenever the recycle space or the polynomial changed.
int Solver::ensure_vc(int kc) {
  if (vc_par == par && vc_updates == updates && vc_k == kc && vc_poly == poly_builds * 4 + poly_prec) return COARSE_OK;
  for (int c = 0; c < kc; ++c) TRY(opA(C[par][c], VC[par][c], nullptr));
  vc_par = par;
  vc_updates = updates;
  vc_k = kc;
  vc_poly = poly_builds * 4 + poly_prec;
  return COARSE_OK;
}

// Step j of a latency-1 pipelined cycle (Sec. 3.5, Alg. "pipe1fgmres" / "pipe1gcrodr", sigma = 0):
// the fused reduction h = [C, V_0..V_j]^H Va[j], ||Va[j]||^2 runs on aux_stream while the product
// w = A Va[j] -> Va[j+1] runs on `stream`; then t = ||Va[j]||^2 - sum |h|^2 (breakdown if negative),
// V[j+1] = Va[j] - [C, V] h and Va[j+1] = w - [VC, Va] h with the same coefficients, the column's
// Givens update, and both divided by h_{j+1,j} = sqrt(t).
int Solver::p1_step(int j, int kc, void* const* tab) {
  const int* stop = &st->stop;
  const int nq = kc + j + 1;
  double* nva = norm2 + 4;
  void* const* at = kc > 0 ? atab[par] : vatab;
  COARSE_CUDA(cudaEventRecord(ev_fork, stream));
  COARSE_CUDA(cudaStreamWaitEvent(aux_stream, ev_fork, 0));
  TRY(launch_multidot(v64, (const void* const*)tab, nq, Va[j], N, h1, nva, partial, counter, stop, aux_stream));
  COARSE_CUDA(cudaEventRecord(ev_join, aux_stream));
  TRY(opA(Va[j], Va[j + 1], stop));
  COARSE_CUDA(cudaStreamWaitEvent(stream, ev_join, 0));
  TRY(launch_p1_prep(st, h1, nva, v64 ? 0x1p-53 : 0x1p-24, stream));
  // the recurrences run whenever t was usable (also on the step whose finalize then stops the cycle)
  TRY(launch_scale(v64, Va[j], nullptr, make_double2(1.0, 0.0), V[j + 1], N, &st->p1_skip, 0, stream));
  TRY(launch_update(v64, (const void* const*)tab, nq, h1, 1, V[j + 1], N, 0, nullptr, nullptr, partial, counter,
                    &st->p1_skip, stream));
  TRY(launch_update(v64, (const void* const*)at, nq, h1, 1, Va[j + 1], N, 0, nullptr, nullptr, partial, counter,
                    &st->p1_skip, stream));
  TRY(launch_step_finalize(st, h1, nullptr, dn, stream));
  TRY(launch_scale(v64, V[j + 1], &st->inv_h, make_double2(1.0, 0.0), V[j + 1], N, &st->j, j + 1, stream));
  return launch_scale(v64, Va[j + 1], &st->inv_h, make_double2(1.0, 0.0), Va[j + 1], N, &st->j, j + 1, stream);
}

// Orthogonalise V[j+1] against [C (kc), V_0..V_j] twice (CGS2, one fused reduction per pass),
// then finalize the Arnoldi column and normalise.
int Solver::arnoldi_step(int j, int kc, void* const* tab) {
  const int* stop = &st->stop;
  const int nq = kc + j + 1;
  void* wv = V[j + 1];
  // pass 1: h1 = Q^H w;  w -= Q h1 fused with pass 2's dots h2 = Q^H w;  w -= Q h2 with ||w||^2
  TRY(launch_multidot(v64, (const void* const*)tab, nq, wv, N, h1, nullptr, partial, counter, stop, stream));
  TRY(launch_update(v64, (const void* const*)tab, nq, h1, 1, wv, N, 2, h2, nullptr, partial, counter, stop, stream));
  TRY(launch_update(v64, (const void* const*)tab, nq, h2, 1, wv, N, 1, nullptr, &st->wnorm2, partial, counter, stop,
                    stream));
  TRY(launch_step_finalize(st, h1, h2, dn, stream));
  // normalise v_{j+1} whenever the finalize of this step ran (st->j == j + 1), also on the step that stops
  return launch_scale(v64, wv, &st->inv_h, make_double2(1.0, 0.0), wv, N, &st->j, j + 1, stream);
}

int Solver::build_poly(const double2* start64, uint64_t seed, int dd) {
  clear_graphs();  // graphs bake host-side chain constants (theta_1 for degree 1)
  ++poly_builds;
  poly_ok = false;
  d = 0;
  if (dd <= 0) { poly_ok = true; return COARSE_OK; }
  if (start64) {
    TRY(launch_copy_to(v64, start64, r, N, stream));
  } else {
    TRY(launch_fill_gaussian((double2*)tmp64, N, seed, stream));
    TRY(launch_copy_to(v64, (const double2*)tmp64, r, N, stream));
  }
  TRY(launch_norm2(v64, r, N, norm2, partial, counter, stream));
  TRY(launch_cycle_init(st, 0, dd, norm2, 0.0, dn.g, stream));
  TRY(launch_scale(v64, r, &st->inv_h, make_double2(1.0, 0.0), V[0], N, nullptr, 0, stream));
  for (int j = 0; j < dd; ++j) {
    cur_tag = j;
    TRY(apply(V[j], V[j + 1], APPLY_PLAIN, nullptr, nullptr, &st->stop));
    TRY(arnoldi_step(j, 0, vtab));
  }
  cur_tag = -1;
  TRY(launch_poly_roots(st, dn, dd, stream));
  TRY(read_state());
  harvest(st_host->j);
  if (st_host->rstatus != 0 || st_host->d <= 0) {
    set_error("polynomial construction failed (harmonic Ritz problem status %d)", st_host->rstatus);
    return COARSE_ERR_BREAKDOWN;
  }
  d = st_host->d;
  theta_host.resize(d);
  COARSE_CUDA(cudaMemcpyAsync(theta_host.data(), dn.theta, sizeof(double2) * d, cudaMemcpyDeviceToHost, stream));
  double2 sc;
  COARSE_CUDA(cudaMemcpyAsync(&sc, dn.polyc + kPolyScale, sizeof(double2), cudaMemcpyDeviceToHost, stream));
  COARSE_CUDA(cudaStreamSynchronize(stream));
  theta1_inv = sc;
  poly_ok = true;
  return COARSE_OK;
}

// Inner solve A e = r (A = D q(D)), e accumulates M * (update).  r and e live in
// this solver's buffers; r holds the initial residual.  Ends when the
// least-squares residual reaches target_abs or after max_cycles cycles.
int Solver::inner(double target_abs, int max_cycles, int m, int kdef, int ulimit, InnerInfo* info) {
  const int* nostop = nullptr;
  TRY(launch_norm2(v64, r, N, norm2, partial, counter, stream));
  for (int cyc = 0; cyc < max_cycles; ++cyc) {
    const int kc = k_cur;
    if (kc > 0) {
      // keep r orthogonal to range(C): e += M U (C^H r), r -= C (C^H r)  (GCRO-DR, Sec. 3.4)
      TRY(launch_multidot(v64, (const void* const*)qtab[par], kc, r, N, dn.ycoef, nullptr, partial, counter, nostop,
                          stream));
      TRY(launch_update(v64, (const void* const*)qtab[par], kc, dn.ycoef, 1, r, N, 1, nullptr, norm2, partial,
                        counter, nostop, stream));
      TRY(launch_combine(v64, (const void* const*)utab[par], kc, dn.ycoef, 1, (void* const*)one_t, 1, 0, N, nostop,
                         stream));
      const void* mt = nullptr;
      TRY(precondition(t, &mt, nostop));
      TRY(launch_axpy(v64, mt, e, make_double2(1.0, 0.0), N, nostop, stream));
    }
    const int steps = kc > 0 ? m - kc : m;
    void* const* tab = kc > 0 ? qtab[par] : vtab;
    // a cycle that is to yield the first recycle space runs all m steps (no least-squares stop)
    const bool extract_full = full_first && kc == 0 && kdef > 0 && updates < ulimit;
    // pipelined cycles (Sec. 3.5): every cycle of pipelined GMRES; the cycles of GCRO-DR that have
    // a recycle space (its first cycle is the classical GMRES cycle)
    p1_active = pipelined && !p1_off && (kdef == 0 || kc > 0);
    if (p1_active) {
      TRY(ensure_p1());
      if (kc > 0) TRY(ensure_vc(kc));
    }
    TRY(launch_cycle_init(st, kc, steps, norm2, extract_full ? 0.0 : target_abs, dn.g, stream));
    TRY(launch_scale(v64, r, &st->inv_h, make_double2(1.0, 0.0), V[0], N, &st->stop, 0, stream));
    if (p1_active) TRY(opA(V[0], Va[0], &st->stop));  // v^a_0 = A v_0
    // Steps go out in chunks; the stop flag of chunk c-1 is read back (async copy +
    // event) while chunk c runs, so at most one chunk of gated launches follows a stop.
    constexpr int kChunk = 4;
    int pending = -1;  // chunk whose flag copy is in flight
    int launched = 0;
    for (int j0 = 0; j0 < steps; j0 += kChunk) {
      const int cnt = steps - j0 < kChunk ? steps - j0 : kChunk;
      launched += cnt;
      TRY(run_chunk(j0, cnt, kc, tab));
      const int slot = (j0 / kChunk) & 1;
      COARSE_CUDA(cudaMemcpyAsync(stop_host + slot, &st->stop, sizeof(int), cudaMemcpyDeviceToHost, stream));
      COARSE_CUDA(cudaEventRecord(chunk_ev[slot], stream));
      if (pending >= 0) {
        COARSE_CUDA(cudaEventSynchronize(chunk_ev[pending]));
        if (stop_host[pending]) break;
      }
      pending = slot;
    }
    cur_tag = -1;
    TRY(read_state());
    const CycleState cs = *st_host;
    harvest(cs.j);
    ++cycles_done;
    matvecs -= (long long)(launched - cs.j) * (d > 1 ? d : 1);  // gated steps did not run
    info->cycles++;
    if (cs.status & ST_NONFINITE) {
      if (p1_active) {
        // Sec. 3.5: the pipelined recurrences never renormalise v^a; after a loss of orthogonality
        // they can grow without bound.  The cycle is dropped (r and e untouched) and the solve goes
        // on with classical cycles, counted as a breakdown.
        info->breakdowns++;
        p1_off = true;
        continue;
      }
      set_error("non-finite value in the Arnoldi process");
      return COARSE_ERR_NONFINITE;
    }
    if (cs.status & ST_ZERO) return COARSE_OK;  // zero residual
    if (cs.status & ST_BREAKDOWN) info->breakdowns++;
    const int j = cs.j;
    info->iterations += j;
    info->last_resid = cs.resid;
    if (j == 0) return COARSE_OK;
    TRY(launch_cycle_solve(st, dn, stream));
    // e += M (U y_U + V y_V)
    void* const* ut = kc > 0 ? utab[par] : vtab;
    TRY(launch_combine(v64, (const void* const*)ut, kc + j, dn.ycoef, 1, (void* const*)one_t, 1, 0,
                       N, nostop, stream));
    const void* mt = nullptr;
    TRY(precondition(t, &mt, nostop));
    TRY(launch_axpy(v64, mt, e, make_double2(1.0, 0.0), N, nostop, stream));
    // r -= V_{j+1} (Hbar y_V)
    TRY(launch_update(v64, (const void* const*)vtab, j + 1, dn.z, 1, r, N, 1, nullptr, norm2, partial, counter, nostop,
                      stream));
    // recycle space (Sec. 3.4): first extraction needs more than k steps; then up to ulimit updates.
    // A pipelined cycle in FP32 / BF16 makes no update: its Hessenberg entries come from
    // t = ||v^a||^2 - sum |h|^2 (Sec. 3.5), whose cancellation leaves them too inexact for the
    // harmonic Ritz update (A U = C degraded to 4e-3 on the twisted-mass lattice); FP64 ones do.
    const bool can = kdef > 0 && updates < ulimit && !(p1_active && !v64) &&
                     ((kc == 0 && j > kdef) || (kc > 0 && j >= 1));
    if (can) {
      for (int c = 0; c < kc; ++c)
        TRY(launch_multidot(v64, (const void* const*)qtab[par], kc + j + 1, U[par][c], N, SW + (size_t)c * ldsw,
                            nullptr, partial, counter, nostop, stream));
      TRY(launch_recycle(st, dn, SW, ldsw, kdef, stream));
      TRY(read_state());
      harvest(1 << 30);
      if (st_host->rstatus == 0) {
        void* const* wt = kc > 0 ? qtab[par] : vtab;
        TRY(launch_combine(v64, (const void* const*)wt, kc + j + 1, dn.coefC, kdef, (void* const*)cnew[par], kdef, 0,
                           N, nostop, stream));
        TRY(launch_combine(v64, (const void* const*)ut, kc + j, dn.coefU, kdef, (void* const*)unew[par], kdef, 0, N,
                           nostop, stream));
        par = 1 - par;
        k_cur = kdef;
        ++updates;
      } else {
        info->recycle_failures++;
      }
    }
    if (cs.resid <= target_abs || (cs.status & ST_LUCKY)) return COARSE_OK;
  }
  return COARSE_OK;
}

// Sec. 3.4: the recycle space satisfies A U_k = C_k and C_k^H C_k = I for the preconditioned
// operator A = D q(D) it was built for.  Both relations are re-evaluated here from the held
// vectors: one application of A per column (the polynomial chain included), one fused
// reduction per column for C^H c_i.
int Solver::recycle_check(double out[4]) {
  out[0] = out[1] = 0.0;
  out[2] = k_cur;
  out[3] = updates;
  if (k_cur == 0 || !vecmem) return COARSE_OK;
  std::vector<double2> g(k_cur);
  for (int c = 0; c < k_cur; ++c) {
    TRY(opA(U[par][c], w, nullptr));
    TRY(launch_axpy(v64, C[par][c], w, make_double2(-1.0, 0.0), N, nullptr, stream));
    TRY(launch_norm2(v64, w, N, norm2, partial, counter, stream));
    TRY(launch_norm2(v64, C[par][c], N, norm2 + 1, partial, counter, stream));
    TRY(launch_multidot(v64, (const void* const*)qtab[par], k_cur, C[par][c], N, h1, nullptr, partial, counter,
                        nullptr, stream));
    double nn[2];
    COARSE_CUDA(cudaMemcpyAsync(nn, norm2, sizeof(nn), cudaMemcpyDeviceToHost, stream));
    COARSE_CUDA(cudaMemcpyAsync(g.data(), h1, sizeof(double2) * k_cur, cudaMemcpyDeviceToHost, stream));
    COARSE_CUDA(cudaStreamSynchronize(stream));
    const double rel = nn[1] > 0.0 ? sqrt(nn[0] / nn[1]) : INFINITY;
    out[0] = fmax(out[0], rel);
    for (int i = 0; i < k_cur; ++i) {
      const double re = g[i].x - (i == c ? 1.0 : 0.0), im = g[i].y;
      out[1] = fmax(out[1], sqrt(re * re + im * im));
    }
  }
  harvest(1 << 30);
  return COARSE_OK;
}

}  // namespace coarse

namespace coarse {

namespace {
double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

Solver* get_solver(coarse_op* op, int prec, int adjoint_system, cudaStream_t stream, int odd_even) {
  // With mu = 0, D_c(-mu) = D_c: the adjoint system reuses the forward solver (polynomial, recycle space).
  const bool separate = adjoint_system && op->mu != 0.0;
  Solver*& slot = odd_even ? (separate ? op->eo_adj_solver[prec] : op->eo_solver[prec])
                           : (separate ? op->adj_solver[prec] : op->solver[prec]);
  if (slot == nullptr) {
    slot = new Solver();
    slot->op = op;
    slot->prec = prec;
    slot->v64 = prec == COARSE_PREC_FP64;
    slot->eo = odd_even;
    slot->N = odd_even ? op->V * op->n / 2 : op->V * op->n;
    slot->tmp64 = op->work64 + (size_t)op->V * op->n;
    slot->mu_eff = separate ? -op->mu : op->mu;
  }
  slot->stream = stream;
  return slot;
}

int solve_column(coarse_op* op, Solver* s, const double2* b64, double2* x64, const coarse_solve_params* p,
                 coarse_solve_info* info, cudaStream_t stream, int mu_sign) {
  const double t0 = now_ms();
  coarse_solve_info inf{};
  const int N = op->V * op->n;
  const double mu_eff = mu_sign * op->mu;
  s->stream = stream;
  double2* r64 = op->work64;
  double hn[2];

  auto residual = [&]() -> int {
    ApplyArgs a = make_apply_args(op, COARSE_PREC_FP64, x64, r64);
    a.z = b64;
    a.coef = op->coef;  // {-1, +1}: r = -D x + b
    a.mu = mu_eff;
    a.mode = APPLY_AXPBY;
    TRY(launch_apply(COARSE_PREC_FP64, op->n, a, stream));
    return launch_norm2(1, r64, N, op->norms, op->red, op->counter, stream);
  };

  if (p->flags & COARSE_ZERO_GUESS) {
    // x = 0: r = b exactly, no stencil launch needed
    COARSE_CUDA(cudaMemsetAsync(x64, 0, sizeof(double2) * (size_t)N, stream));
    COARSE_CUDA(cudaMemcpyAsync(r64, b64, sizeof(double2) * (size_t)N, cudaMemcpyDeviceToDevice, stream));
    TRY(launch_norm2(1, r64, N, op->norms, op->red, op->counter, stream));
  } else {
    TRY(residual());
  }
  TRY(launch_norm2(1, b64, N, op->norms + 1, op->red, op->counter, stream));
  COARSE_CUDA(cudaMemcpyAsync(hn, op->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  COARSE_CUDA(cudaStreamSynchronize(stream));
  const double bn = sqrt(hn[1]);
  double rn = sqrt(hn[0]);
  if (!isfinite(bn) || !isfinite(rn)) {
    set_error("non-finite right-hand side or initial guess");
    inf.status = COARSE_ERR_NONFINITE;
    if (info) *info = inf;
    return COARSE_ERR_NONFINITE;
  }
  if (bn == 0.0) {
    COARSE_CUDA(cudaMemsetAsync(x64, 0, sizeof(double2) * (size_t)N, stream));
    COARSE_CUDA(cudaStreamSynchronize(stream));
    inf.rel_residual = 0.0;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    return COARSE_OK;
  }
  const int m = p->m;
  const int k = p->defl_k;
  const int dd = p->poly_degree;
  float2* eo_full = nullptr;  // odd-even: full-length FP32 residual / correction, then its halves
  float2 *eo_re = nullptr, *eo_ro = nullptr, *eo_to = nullptr, *eo_eo = nullptr;
  if (s->eo) {
    TRY(eo_prepare(op, mu_eff, stream));
    if (!op->eo_scratch && cudaMalloc(&op->eo_scratch, sizeof(float2) * 3 * (size_t)N) != cudaSuccess) {
      cudaGetLastError();
      op->eo_scratch = nullptr;
      set_error("odd-even: scratch allocation failed");
      return COARSE_ERR_OOM;
    }
    eo_full = (float2*)op->eo_scratch;
    eo_re = eo_full + N;
    eo_ro = eo_re + N / 2;
    eo_to = eo_ro + N / 2;
    eo_eo = eo_to + N / 2;
  }
  TRY(s->ensure(m, k, dd > 0 ? dd : 1));
  s->poly_prec = ((p->flags & COARSE_POLY_BF16) && s->prec == COARSE_PREC_FP32 && op->blk[COARSE_PREC_BF16].ptr)
                     ? COARSE_PREC_BF16
                     : s->prec;
  if ((p->flags & COARSE_RESET_RECYCLE) || s->rec_poly_prec != s->poly_prec) {
    // the recycle space spans C = A q(A) U for one fixed q: drop it when q's blocks change
    s->k_cur = 0;
    s->updates = 0;
  }
  s->rec_poly_prec = s->poly_prec;
  const long long mv0 = s->matvecs;
  const long long launches0 = launches_so_far();
  s->time_apply = (p->flags & COARSE_TIME_APPLY) != 0;
  s->full_first = (p->flags & COARSE_RECYCLE_FULL_CYCLE) != 0;
  s->pipelined = (p->flags & COARSE_PIPELINED) != 0;
  s->apply_ms = 0.0;
  s->apply_bytes = 0.0;
  s->apply_count = 0;
  for (int q = 0; q < 3; ++q) {
    s->prec_ms[q] = s->prec_bytes[q] = 0.0;
    s->prec_count[q] = 0;
  }
  if (!s->poly_ok || (p->flags & COARSE_REBUILD_POLY) || s->d_cap < dd || (dd > 0 && s->d == 0) ||
      (dd == 0 && s->d != 0)) {
    const double ts = now_ms();
    TRY(s->build_poly((const double2*)p->poly_start, p->seed, dd));
    inf.setup_ms = now_ms() - ts;
  }
  int rc = COARSE_OK;
  double rel = rn / bn;
  int stall = 0;
  s->p1_off = false;
  double2* xkeep = static_cast<double2*>(s->tmp64);  // x before a pipelined refinement step
  while (rel > p->tol && inf.ir_steps < p->max_ir) {
    InnerInfo ii;
    const bool p1_step_now = s->pipelined && !s->p1_off;
    // relative reduction the inner solve is asked for (the FP64 path solves to the final tolerance)
    const double want = s->v64 ? 0.5 * p->tol * bn / rn : fmax(p->inner_tol, 0.5 * p->tol * bn / rn);
    if (p1_step_now)
      COARSE_CUDA(cudaMemcpyAsync(xkeep, x64, sizeof(double2) * (size_t)N, cudaMemcpyDeviceToDevice, stream));
    COARSE_CUDA(cudaMemsetAsync(s->e, 0, (s->v64 ? sizeof(double2) : sizeof(float2)) * (size_t)N, stream));
    if (s->v64) {
      COARSE_CUDA(cudaMemcpyAsync(s->r, r64, sizeof(double2) * (size_t)N, cudaMemcpyDeviceToDevice, stream));
      TRY(s->inner(0.5 * p->tol * bn, p->max_restarts, m, k, p->recycle_updates, &ii));
      TRY(launch_axpy(1, s->e, x64, make_double2(1.0, 0.0), N, nullptr, stream));
    } else if (s->eo) {
      // Sec. 2 / Sec. 3.2: solve S e_e = D_ee^{-1} (r_e - D_eo D_oo^{-1} r_o), then
      // e_o = D_oo^{-1} (r_o - D_oe e_e) = t_o - D_oo^{-1} D_oe e_e with t_o = D_oo^{-1} r_o
      TRY(launch_to_low(r64, op->norms, eo_full, N, stream));
      TRY(launch_eo_split(0, eo_full, op->eo_sites, op->V, op->n, eo_re, eo_ro, stream));
      EoArgs a{};
      a.blocks = op->blk[s->prec].ptr;
      a.inv = op->inv[eo_sign(op, mu_eff)][s->prec].ptr;
      a.rec = op->eo_rec;
      a.err = op->apply_cnt + op->V;
      a.V = op->V;
      a.mode = APPLY_PLAIN;
      a.out_par = 1;  // t_o = D_oo^{-1} r_o
      a.z = eo_ro;
      a.y = eo_to;
      TRY(launch_eo_half(s->prec, op->n, a, stream));
      a.out_par = 0;  // rhs = D_ee^{-1} (r_e - D_eo t_o)
      a.v = eo_to;
      a.z = eo_re;
      a.y = s->r;
      TRY(launch_eo_half(s->prec, op->n, a, stream));
      const double target = fmax(p->inner_tol, 0.5 * p->tol * bn / rn);
      TRY(s->inner(target, p->max_restarts, m, k, p->recycle_updates, &ii));
      a.out_par = 1;  // e_o = t_o - D_oo^{-1} D_oe e_e
      a.v = s->e;
      a.z = nullptr;
      a.base = eo_to;
      a.y = eo_eo;
      TRY(launch_eo_half(s->prec, op->n, a, stream));
      TRY(launch_eo_merge(0, s->e, eo_eo, op->eo_sites, op->V, op->n, eo_full, stream));
      TRY(launch_add_low(x64, op->norms, eo_full, N, stream));
    } else {
      TRY(launch_to_low(r64, op->norms, (float2*)s->r, N, stream));
      const double target = fmax(p->inner_tol, 0.5 * p->tol * bn / rn);
      TRY(s->inner(target, p->max_restarts, m, k, p->recycle_updates, &ii));
      TRY(launch_add_low(x64, op->norms, (const float2*)s->e, N, stream));
    }
    inf.ir_steps++;
    inf.cycles += ii.cycles;
    inf.iterations += ii.iterations;
    inf.breakdowns += ii.breakdowns;
    TRY(residual());
    COARSE_CUDA(cudaMemcpyAsync(hn, op->norms, sizeof(double), cudaMemcpyDeviceToHost, stream));
    COARSE_CUDA(cudaStreamSynchronize(stream));
    double rn_new = sqrt(hn[0]);
    if (p1_step_now && !(rn_new < rn)) {
      // Sec. 3.5: the pipelined recurrences can lose orthogonality without t turning negative;
      // a refinement step that did not lower the true residual is undone, and this solve goes on
      // with classical cycles (counted as a breakdown)
      COARSE_CUDA(cudaMemcpyAsync(x64, xkeep, sizeof(double2) * (size_t)N, cudaMemcpyDeviceToDevice, stream));
      TRY(residual());
      COARSE_CUDA(cudaMemcpyAsync(hn, op->norms, sizeof(double), cudaMemcpyDeviceToHost, stream));
      COARSE_CUDA(cudaStreamSynchronize(stream));
      rn_new = sqrt(hn[0]);
      s->p1_off = true;
      inf.breakdowns++;
      rn = rn_new;
      rel = rn / bn;
      continue;
    }
    if (p1_step_now && rn_new > sqrt(want) * rn) {
      // a pipelined step that lowered the true residual by less than the square root of what its
      // inner solve reported (the recurrence's residual estimate has drifted from the true one) is
      // kept, and the solve goes on with classical cycles (counted as a breakdown)
      s->p1_off = true;
      inf.breakdowns++;
    }
    if (!isfinite(rn_new)) {
      set_error("non-finite residual during refinement");
      rc = COARSE_ERR_NONFINITE;
      break;
    }
    stall = (rn_new > 0.5 * rn) ? stall + 1 : 0;
    rn = rn_new;
    rel = rn / bn;
    if (stall >= 3) break;
  }
  COARSE_CUDA(cudaStreamSynchronize(stream));
  s->harvest(1 << 30);
  s->time_apply = false;
  inf.apply_ms = s->apply_ms;
  inf.apply_bytes = s->apply_bytes;
  inf.apply_count = (int)s->apply_count;
  for (int q = 0; q < 3; ++q) {
    inf.apply_ms_prec[q] = s->prec_ms[q];
    inf.apply_bytes_prec[q] = s->prec_bytes[q];
    inf.apply_count_prec[q] = (int)s->prec_count[q];
  }
  inf.kernel_launches = (int)(launches_so_far() - launches0);
  inf.matvecs = (int)(s->matvecs - mv0);
  inf.recycle_updates = s->updates;
  inf.rel_residual = rel;
  if (rc == COARSE_OK && rel > p->tol) {
    set_error("tolerance %.3e not reached: relative residual %.3e after %d refinement steps", p->tol, rel,
              inf.ir_steps);
    rc = COARSE_ERR_NOT_CONVERGED;
  }
  inf.status = rc;
  inf.solve_ms = now_ms() - t0;
  if (info) *info = inf;
  return rc;
}

}  // namespace coarse
