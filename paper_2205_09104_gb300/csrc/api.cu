// C ABI of the coarse library (declarations and argument contracts in include/coarse.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "common.cuh"
#include "oddeven.cuh"
#include "solver.cuh"

namespace coarse {

namespace {
thread_local std::string g_error;
std::atomic<long long> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return COARSE_ERR_CUDA;
}

namespace {

#define TRY(call)                     \
  do {                                \
    int _rc = (call);                 \
    if (_rc != COARSE_OK) return _rc; \
  } while (0)

bool valid_nv(int nv) { return nv == 8 || nv == 16 || nv == 24; }

template <class T>
int dmalloc(T** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes == 0 ? 1 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return COARSE_ERR_OOM;
  }
  return COARSE_OK;
}

void free_op(coarse_op* op) {
  if (!op) return;
  cudaDeviceSynchronize();
  for (int p = 0; p < 3; ++p) {
    delete op->solver[p];
    delete op->adj_solver[p];
    if (op->blk[p].ptr) cudaFree(op->blk[p].ptr);
  }
  if (op->mrhs.ptr) cudaFree(op->mrhs.ptr);
  for (int p = 0; p < 3; ++p) {
    delete op->eo_solver[p];
    delete op->eo_adj_solver[p];
    for (int sg = 0; sg < 2; ++sg)
      if (op->inv[sg][p].ptr) cudaFree(op->inv[sg][p].ptr);
  }
  if (op->eo_sites) cudaFree(op->eo_sites);
  if (op->eo_half) cudaFree(op->eo_half);
  if (op->eo_rec) cudaFree(op->eo_rec);
  if (op->eo_scratch) cudaFree(op->eo_scratch);
  if (op->mrhs_x.ptr) cudaFree(op->mrhs_x.ptr);
  if (op->umma.ptr) cudaFree(op->umma.ptr);
  if (op->nb) cudaFree(op->nb);
  if (op->work64) cudaFree(op->work64);
  if (op->red) cudaFree(op->red);
  if (op->apply_scratch) cudaFree(op->apply_scratch);
  if (op->apply_cnt) cudaFree(op->apply_cnt);
  delete op;
}

int check_ptr(const void* p, const char* name) {
  if (p == nullptr) {
    set_error("%s is NULL", name);
    return COARSE_ERR_INVALID_ARG;
  }
  return COARSE_OK;
}

int ingest(coarse_op* op, const void* self_b, const void* hop_b, uint32_t flags, cudaStream_t s) {
  const int gamma5_only = (flags & COARSE_ASSUME_GAMMA5) ? 1 : 0;
  if (!gamma5_only) {
    TRY(launch_gamma5_defect((const double2*)self_b, (const double2*)hop_b, op->V, op->n, op->nb, op->norms + 2, s));
    double h[2];
    COARSE_CUDA(cudaMemcpyAsync(h, op->norms + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
    COARSE_CUDA(cudaStreamSynchronize(s));
    if (!isfinite(h[0]) || !isfinite(h[1])) {
      set_error("coarse_op_create: non-finite block entries");
      return COARSE_ERR_NONFINITE;
    }
    if (h[0] > 1e-10 * h[1]) {
      set_error("blocks violate sigma3 D_c sigma3 = D_c^H: max defect %.3e, max entry %.3e", h[0], h[1]);
      return COARSE_ERR_NOT_GAMMA5;
    }
  }
  TRY(launch_ingest((const double2*)self_b, (const double2*)hop_b, gamma5_only, op->V, op->n, op->nb,
                    op->blk[0].ptr, op->blk[1].ptr, op->blk[2].ptr, s));
  TRY(launch_pack_mrhs(op, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  return COARSE_OK;
}

int validate_solve(const coarse_op* op, const void* b, const void* x, int nrhs, const coarse_solve_params* p) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(b, "b"));
  TRY(check_ptr(x, "x"));
  TRY(check_ptr(p, "params"));
  if (nrhs < 1) { set_error("nrhs = %d < 1", nrhs); return COARSE_ERR_INVALID_ARG; }
  if (p->m < 2 || p->m > kMaxDense) { set_error("restart length m = %d outside [2, %d]", p->m, kMaxDense); return COARSE_ERR_INVALID_ARG; }
  if (p->defl_k < 0 || p->defl_k > kMaxK || (p->defl_k > 0 && p->defl_k >= p->m)) {
    set_error("deflation k = %d must satisfy 0 <= k < m and k <= %d", p->defl_k, kMaxK);
    return COARSE_ERR_INVALID_ARG;
  }
  if (p->poly_degree < 0 || p->poly_degree > kMaxPoly) {
    set_error("poly_degree = %d outside [0, %d]", p->poly_degree, kMaxPoly);
    return COARSE_ERR_INVALID_ARG;
  }
  if (p->precision < 0 || p->precision > 2) { set_error("unknown precision %d", p->precision); return COARSE_ERR_INVALID_ARG; }
  if (!op->blk[p->precision].ptr) {
    set_error("precision %d was not enabled in coarse_op_desc.precisions", p->precision);
    return COARSE_ERR_INVALID_ARG;
  }
  if (!(p->tol > 0.0) || p->max_restarts < 1 || p->max_ir < 1 || p->recycle_updates < 0) {
    set_error("need tol > 0, max_restarts >= 1, max_ir >= 1, recycle_updates >= 0");
    return COARSE_ERR_INVALID_ARG;
  }
  if (p->precision != COARSE_PREC_FP64 && !(p->inner_tol > 0.0 && p->inner_tol < 1.0)) {
    set_error("inner_tol = %g must lie in (0, 1)", p->inner_tol);
    return COARSE_ERR_INVALID_ARG;
  }
  return COARSE_OK;
}

int apply_impl(const coarse_op* op, const void* x, void* y, int nrhs, int precision, void* stream, int adjoint) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(x, "x"));
  TRY(check_ptr(y, "y"));
  if (precision < 0 || precision > 2 || !op->blk[precision].ptr) {
    set_error("precision %d not available on this operator", precision);
    return COARSE_ERR_INVALID_ARG;
  }
  if (nrhs < 1 || nrhs > op->max_nrhs) {
    set_error("nrhs = %d outside [1, max_nrhs = %d]", nrhs, op->max_nrhs);
    return COARSE_ERR_INVALID_ARG;
  }
  if (x == y) { set_error("x and y must not overlap"); return COARSE_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  if (nrhs > 1 && precision == COARSE_PREC_BF16) return launch_apply_mrhs_bf16(op, x, y, nrhs, adjoint, s);
  const size_t esz = precision == COARSE_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t col = esz * (size_t)op->V * op->n;
  for (int c = 0; c < nrhs; ++c) {
    ApplyArgs a = make_apply_args(op, precision, (const char*)x + c * col, (char*)y + c * col);
    a.mu = adjoint ? -op->mu : op->mu;
    a.adjoint = adjoint;
    TRY(launch_apply(precision, op->n, a, s));
  }
  return COARSE_OK;
}

}  // namespace

// Error flag of the operator's staged stencil kernels (raised when one of their bounded waits ran
// out, leaving that launch's output incomplete): read and clear it; COARSE_ERR_TIMEOUT if raised.
int take_stencil_flag(const coarse_op* op, cudaStream_t s) {
  int h = 0;
  COARSE_CUDA(cudaMemcpyAsync(&h, op->apply_cnt + op->V, sizeof(int), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  if (h == 0) return COARSE_OK;
  COARSE_CUDA(cudaMemsetAsync(op->apply_cnt + op->V, 0, sizeof(int), s));
  set_error("a bounded wait of a staged stencil kernel ran out; the results since the last check are invalid");
  return COARSE_ERR_TIMEOUT;
}

namespace {

int solve_impl(coarse_op* op, const void* b, void* x, int nrhs, const coarse_solve_params* p,
               coarse_solve_info* info, void* stream, int adjoint) {
  TRY(validate_solve(op, b, x, nrhs, p));
  // odd-even reduction: FP32/BF16 inner precision (FP64 solves keep the full operator); odd
  // extents cannot be split and are an error
  int eo = (p->flags & COARSE_ODD_EVEN) ? 1 : 0;
  if (eo && !op->eo_sites) {
    set_error("COARSE_ODD_EVEN needs even lattice extents");
    return COARSE_ERR_INVALID_ARG;
  }
  if (p->precision == COARSE_PREC_FP64) eo = 0;
  cudaStream_t s = (cudaStream_t)stream;
  COARSE_CUDA(cudaSetDevice(op->device));
  Solver* sv = get_solver(op, p->precision, adjoint, s, eo);
  const size_t N = (size_t)op->V * op->n;
  int worst = COARSE_OK;
  for (int c = 0; c < nrhs; ++c) {
    const double2* bc = (const double2*)b + c * N;
    double2* xc = (double2*)x + c * N;
    coarse_solve_info inf{};
    int rc;
    if (!adjoint) {
      rc = solve_column(op, sv, bc, xc, p, &inf, s, +1);
    } else {
      // D^H lambda = c  <=>  D(-mu) (sigma3 lambda) = sigma3 c
      double2* sb = op->work64 + 2 * N;
      TRY(launch_sigma3(1, bc, sb, op->n, op->V, s));
      if (!(p->flags & COARSE_ZERO_GUESS)) TRY(launch_sigma3(1, xc, xc, op->n, op->V, s));
      rc = solve_column(op, sv, sb, xc, p, &inf, s, -1);
      TRY(launch_sigma3(1, xc, xc, op->n, op->V, s));
      COARSE_CUDA(cudaStreamSynchronize(s));
    }
    if (info) info[c] = inf;
    if (rc != COARSE_OK && rc != COARSE_ERR_NOT_CONVERGED) return rc;
    if (rc != COARSE_OK) worst = rc;
  }
  TRY(take_stencil_flag(op, s));
  return worst;
}

}  // namespace
}  // namespace coarse

using namespace coarse;

extern "C" {

int coarse_op_create(const coarse_op_desc* d, const void* self_blocks, const void* hop_blocks, void* stream,
                     coarse_op** out) {
  TRY(check_ptr(d, "desc"));
  TRY(check_ptr(self_blocks, "self_blocks"));
  TRY(check_ptr(hop_blocks, "hop_blocks"));
  TRY(check_ptr(out, "out"));
  *out = nullptr;
  for (int mu = 0; mu < 4; ++mu)
    if (d->dims[mu] < 2) {
      set_error("dims[%d] = %d < 2", mu, d->dims[mu]);
      return COARSE_ERR_INVALID_ARG;
    }
  if (!valid_nv(d->nv)) {
    set_error("nv = %d unsupported (8, 16 or 24)", d->nv);
    return COARSE_ERR_INVALID_ARG;
  }
  if (d->max_nrhs < 1 || d->max_nrhs > 64) {
    set_error("max_nrhs = %d outside [1, 64]", d->max_nrhs);
    return COARSE_ERR_INVALID_ARG;
  }
  const long long Vll = (long long)d->dims[0] * d->dims[1] * d->dims[2] * d->dims[3];
  if (Vll * 2 * d->nv > (1ll << 30)) {
    set_error("lattice too large: V*n = %lld", Vll * 2 * d->nv);
    return COARSE_ERR_INVALID_ARG;
  }
  if (!isfinite(d->mu)) {
    set_error("mu is not finite");
    return COARSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  coarse_op* op = new coarse_op();
  cudaGetDevice(&op->device);
  memcpy(op->dims, d->dims, sizeof(op->dims));
  op->V = (int)Vll;
  op->nv = d->nv;
  op->n = 2 * d->nv;
  op->mu = d->mu;
  op->max_nrhs = d->max_nrhs;
  op->precisions = d->precisions | 1u;
  const size_t N = (size_t)op->V * op->n;
  // neighbour table
  std::vector<int> nb((size_t)op->V * 8);
  const int* L = op->dims;
  for (int x = 0; x < op->V; ++x) {
    int c[4], r = x;
    for (int mu = 0; mu < 4; ++mu) { c[mu] = r % L[mu]; r /= L[mu]; }
    for (int dd = 0; dd < 8; ++dd) {
      int cc[4] = {c[0], c[1], c[2], c[3]};
      const int mu = dd % 4;
      cc[mu] = (cc[mu] + (dd < 4 ? 1 : L[mu] - 1)) % L[mu];
      nb[(size_t)x * 8 + dd] = cc[0] + L[0] * (cc[1] + L[1] * (cc[2] + L[2] * cc[3]));
    }
  }
  int rc = COARSE_OK;
  const size_t nblk = (size_t)op->V * 5 * op->n * op->n;
  const size_t esz[3] = {sizeof(double2), sizeof(float2), sizeof(cbf16)};
#define CREATE_TRY(call)                    \
  do {                                      \
    rc = (call);                            \
    if (rc != COARSE_OK) { free_op(op); return rc; } \
  } while (0)
  CREATE_TRY(dmalloc(&op->nb, nb.size() * sizeof(int)));
  // odd-even site lists (every extent even: each hop joins opposite parities)
  std::vector<int> eo_sites, eo_half;
  std::vector<int4> eo_rec;
  if (L[0] % 2 == 0 && L[1] % 2 == 0 && L[2] % 2 == 0 && L[3] % 2 == 0) {
    eo_sites.resize(op->V);
    eo_half.resize(op->V);
    int ne = 0, no = op->V / 2;
    for (int x = 0; x < op->V; ++x) {
      int c[4], r = x;
      for (int mu = 0; mu < 4; ++mu) { c[mu] = r % L[mu]; r /= L[mu]; }
      const bool odd = (c[0] + c[1] + c[2] + c[3]) & 1;
      const int q = odd ? no++ : ne++;
      eo_sites[q] = x;
      eo_half[x] = odd ? q - op->V / 2 : q;
    }
    CREATE_TRY(dmalloc(&op->eo_sites, eo_sites.size() * sizeof(int)));
    CREATE_TRY(dmalloc(&op->eo_half, eo_half.size() * sizeof(int)));
    eo_rec.resize((size_t)op->V * 4);
    for (int q = 0; q < op->V; ++q) {
      const int x = eo_sites[q];
      for (int mu = 0; mu < 4; ++mu) {
        const int f = nb[(size_t)x * 8 + mu], b = nb[(size_t)x * 8 + 4 + mu];
        eo_rec[(size_t)q * 4 + mu] = make_int4(eo_half[f], b, eo_half[b], x);
      }
    }
    CREATE_TRY(dmalloc(&op->eo_rec, eo_rec.size() * sizeof(int4)));
  }
  for (int p = 0; p < 3; ++p) {
    if (!(op->precisions & (1u << p))) continue;
    op->blk[p].bytes = nblk * esz[p];
    CREATE_TRY(dmalloc((char**)&op->blk[p].ptr, op->blk[p].bytes));
  }
  if ((op->precisions & (1u << COARSE_PREC_BF16)) && op->max_nrhs > 1) {
    op->mrhs.bytes = nblk * sizeof(cbf16);
    CREATE_TRY(dmalloc((char**)&op->mrhs.ptr, op->mrhs.bytes));
    // 12 columns as mma.sync fragments (12 N BF16 pairs); where the tcgen05 kernel exists,
    // also 16 columns as its two B-operand variants (32 N)
    const bool tc = op->n == 32 || op->n == 48;
    op->mrhs_x.bytes = (tc ? 32 : 12) * N * sizeof(cbf16);
    CREATE_TRY(dmalloc((char**)&op->mrhs_x.ptr, op->mrhs_x.bytes));
    if (tc) {
      op->umma.bytes = nblk * sizeof(cbf16);
      CREATE_TRY(dmalloc((char**)&op->umma.ptr, op->umma.bytes));
    }
  }
  CREATE_TRY(dmalloc(&op->work64, 3 * N * sizeof(double2)));
  CREATE_TRY(dmalloc((char**)&op->apply_scratch, 5 * N * sizeof(double2)));
  CREATE_TRY(dmalloc(&op->apply_cnt, ((size_t)op->V + 4) * sizeof(int)));
  CREATE_TRY(dmalloc((char**)&op->red, (2 * 304 + 64) * sizeof(double) + 64));
  op->norms = op->red + 2 * 304;
  op->coef = (double2*)(op->norms + 8);
  op->counter = (unsigned*)(op->coef + 2);
  const double2 cst[2] = {make_double2(-1.0, 0.0), make_double2(1.0, 0.0)};
  if ((op->eo_sites &&
       (cudaMemcpyAsync(op->eo_sites, eo_sites.data(), eo_sites.size() * sizeof(int), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(op->eo_half, eo_half.data(), eo_half.size() * sizeof(int), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(op->eo_rec, eo_rec.data(), eo_rec.size() * sizeof(int4), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)) ||
      cudaMemcpyAsync(op->nb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(op->red, 0, (2 * 304 + 64) * sizeof(double) + 64, s) != cudaSuccess ||
      cudaMemsetAsync(op->apply_cnt, 0, ((size_t)op->V + 4) * sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(op->coef, cst, sizeof(cst), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cuda_fail(cudaGetLastError(), "coarse_op_create copies");
    free_op(op);
    return COARSE_ERR_CUDA;
  }
  CREATE_TRY(ingest(op, self_blocks, hop_blocks, d->flags, s));
#undef CREATE_TRY
  *out = op;
  return COARSE_OK;
}

int coarse_op_update(coarse_op* op, const void* self_blocks, const void* hop_blocks, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(self_blocks, "self_blocks"));
  TRY(check_ptr(hop_blocks, "hop_blocks"));
  TRY(ingest(op, self_blocks, hop_blocks, 0, (cudaStream_t)stream));
  op->inv_ok[0] = op->inv_ok[1] = 0;
  for (int p = 0; p < 3; ++p) {
    if (op->solver[p]) op->solver[p]->invalidate();
    if (op->adj_solver[p]) op->adj_solver[p]->invalidate();
    if (op->eo_solver[p]) op->eo_solver[p]->invalidate();
    if (op->eo_adj_solver[p]) op->eo_adj_solver[p]->invalidate();
  }
  return COARSE_OK;
}

void coarse_op_destroy(coarse_op* op) { free_op(op); }

int coarse_apply(const coarse_op* op, const void* x, void* y, int nrhs, int precision, void* stream) {
  return apply_impl(op, x, y, nrhs, precision, stream, 0);
}

int coarse_apply_adjoint(const coarse_op* op, const void* x, void* y, int nrhs, int precision, void* stream) {
  return apply_impl(op, x, y, nrhs, precision, stream, 1);
}

int coarse_schur_apply(coarse_op* op, const void* x, void* y, int precision, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(x, "x"));
  TRY(check_ptr(y, "y"));
  if (precision < 0 || precision > 2 || !op->blk[precision].ptr) {
    set_error("precision %d not available on this operator", precision);
    return COARSE_ERR_INVALID_ARG;
  }
  if (x == y) { set_error("x and y must not overlap"); return COARSE_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  TRY(eo_prepare(op, op->mu, s));
  // odd-site intermediate: the third FP64 work vector (large enough for V/2 * n complex128)
  void* t = op->work64 + 2 * (size_t)op->V * op->n;
  return launch_eo_schur(op, precision, op->mu, x, y, t, APPLY_PLAIN, nullptr, nullptr, nullptr, s);
}

int coarse_residual(const coarse_op* op, const void* b, const void* x, void* r, double* norms_host, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(b, "b"));
  TRY(check_ptr(x, "x"));
  TRY(check_ptr(r, "r"));
  TRY(check_ptr(norms_host, "norms_host"));
  if (r == x || r == b) { set_error("r must not alias b or x"); return COARSE_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  const int N = op->V * op->n;
  ApplyArgs a = make_apply_args(op, COARSE_PREC_FP64, x, r);
  a.z = b;
  a.coef = op->coef;
  a.mode = APPLY_AXPBY;
  TRY(launch_apply(COARSE_PREC_FP64, op->n, a, s));
  TRY(launch_norm2(1, r, N, op->norms + 4, op->red, op->counter, s));
  TRY(launch_norm2(1, b, N, op->norms + 5, op->red, op->counter, s));
  double h[2];
  COARSE_CUDA(cudaMemcpyAsync(h, op->norms + 4, sizeof(h), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  norms_host[0] = sqrt(h[0]);
  norms_host[1] = sqrt(h[1]);
  return take_stencil_flag(op, s);
}

int coarse_solve(coarse_op* op, const void* b, void* x, int nrhs, const coarse_solve_params* params,
                 coarse_solve_info* info_host, void* stream) {
  return solve_impl(op, b, x, nrhs, params, info_host, stream, 0);
}

int coarse_solve_adjoint(coarse_op* op, const void* b, void* x, int nrhs, const coarse_solve_params* params,
                         coarse_solve_info* info_host, void* stream) {
  return solve_impl(op, b, x, nrhs, params, info_host, stream, 1);
}

int coarse_block_grad(const coarse_op* op, const void* lambda, const void* x, void* g_self, void* g_hop,
                      int hop_dirs, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(lambda, "lambda"));
  TRY(check_ptr(x, "x"));
  TRY(check_ptr(g_self, "g_self"));
  TRY(check_ptr(g_hop, "g_hop"));
  if (hop_dirs != 8 && hop_dirs != 4) {
    set_error("hop_dirs = %d (8: canonical layout, 4: gamma5-compressed)", hop_dirs);
    return COARSE_ERR_INVALID_ARG;
  }
  return launch_block_grad((const double2*)lambda, (const double2*)x, op->nb, op->V, op->n, hop_dirs,
                           (double2*)g_self, (double2*)g_hop, (cudaStream_t)stream);
}

namespace {
Solver* held_solver(coarse_op* op, int precision, int odd_even, int adjoint) {
  const bool separate = adjoint && op->mu != 0.0;
  return odd_even ? (separate ? op->eo_adj_solver[precision] : op->eo_solver[precision])
                  : (separate ? op->adj_solver[precision] : op->solver[precision]);
}
}  // namespace

int coarse_recycle_check(coarse_op* op, int precision, int odd_even, int adjoint, double* out_host, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(out_host, "out_host"));
  if (precision < 0 || precision > 2) { set_error("unknown precision %d", precision); return COARSE_ERR_INVALID_ARG; }
  for (int i = 0; i < 4; ++i) out_host[i] = 0.0;
  Solver* s = held_solver(op, precision, odd_even, adjoint);
  if (!s) return COARSE_OK;
  COARSE_CUDA(cudaSetDevice(op->device));
  s->stream = (cudaStream_t)stream;
  TRY(s->recycle_check(out_host));
  return take_stencil_flag(op, (cudaStream_t)stream);
}

int coarse_recycle_get(coarse_op* op, int precision, int odd_even, int adjoint, void* u, void* c, int cap, int* k,
                       void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(k, "k"));
  if (precision < 0 || precision > 2) { set_error("unknown precision %d", precision); return COARSE_ERR_INVALID_ARG; }
  *k = 0;
  Solver* s = held_solver(op, precision, odd_even, adjoint);
  if (!s || s->k_cur == 0 || !s->vecmem) return COARSE_OK;
  if (cap < s->k_cur) {
    set_error("cap = %d is below the %d recycle vectors held", cap, s->k_cur);
    return COARSE_ERR_INVALID_ARG;
  }
  TRY(check_ptr(u, "u"));
  TRY(check_ptr(c, "c"));
  COARSE_CUDA(cudaSetDevice(op->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t col = (s->v64 ? sizeof(double2) : sizeof(float2)) * (size_t)s->N;
  for (int i = 0; i < s->k_cur; ++i) {
    COARSE_CUDA(cudaMemcpyAsync((char*)u + i * col, s->U[s->par][i], col, cudaMemcpyDeviceToDevice, st));
    COARSE_CUDA(cudaMemcpyAsync((char*)c + i * col, s->C[s->par][i], col, cudaMemcpyDeviceToDevice, st));
  }
  COARSE_CUDA(cudaStreamSynchronize(st));
  *k = s->k_cur;
  return COARSE_OK;
}

int coarse_recycle_set(coarse_op* op, int precision, int odd_even, int adjoint, const void* u, const void* c, int k,
                       int updates, void* stream) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  if (precision < 0 || precision > 2) { set_error("unknown precision %d", precision); return COARSE_ERR_INVALID_ARG; }
  Solver* s = held_solver(op, precision, odd_even, adjoint);
  if (!s || !s->vecmem || s->k_cap < k || k < 0) {
    set_error("coarse_recycle_set: no solver of this system with room for k = %d recycle vectors (solve once "
              "with defl_k = %d first)", k, k);
    return COARSE_ERR_INVALID_ARG;
  }
  if (k > 0) {
    TRY(check_ptr(u, "u"));
    TRY(check_ptr(c, "c"));
  }
  COARSE_CUDA(cudaSetDevice(op->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t col = (s->v64 ? sizeof(double2) : sizeof(float2)) * (size_t)s->N;
  for (int i = 0; i < k; ++i) {
    COARSE_CUDA(cudaMemcpyAsync(s->U[s->par][i], (const char*)u + i * col, col, cudaMemcpyDeviceToDevice, st));
    COARSE_CUDA(cudaMemcpyAsync(s->C[s->par][i], (const char*)c + i * col, col, cudaMemcpyDeviceToDevice, st));
  }
  COARSE_CUDA(cudaStreamSynchronize(st));
  s->k_cur = k;
  s->updates = updates < 0 ? 0 : updates;
  s->rec_poly_prec = s->poly_prec;
  s->vc_par = -1;
  return COARSE_OK;
}

int coarse_op_poly(const coarse_op* op, int precision, double* theta_host, int cap, int* d) {
  if (!op) { set_error("op is NULL"); return COARSE_ERR_INVALID_ARG; }
  TRY(check_ptr(d, "d"));
  if (precision < 0 || precision > 2) { set_error("unknown precision %d", precision); return COARSE_ERR_INVALID_ARG; }
  const Solver* s = op->solver[precision];
  if (!(s && s->poly_ok && s->d > 0) && op->eo_solver[precision] && op->eo_solver[precision]->poly_ok)
    s = op->eo_solver[precision];  // only odd-even solves have run: report their polynomial (of B^-1 D_c)
  *d = (s && s->poly_ok) ? s->d : 0;
  if (theta_host && s) {
    for (int i = 0; i < *d && i < cap; ++i) {
      theta_host[2 * i] = s->theta_host[i].x;
      theta_host[2 * i + 1] = s->theta_host[i].y;
    }
  }
  return COARSE_OK;
}

const char* coarse_last_error(void) { return g_error.c_str(); }

const char* coarse_version(void) { return "coarse-gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
