// coarse_residual_noalloc: the FP64 residual r = b - D_c x and its norms with every
// piece of scratch memory in one static device array instead of memory owned by the
// operator handle, for callers that must not allocate during the call.
#include <mutex>

#include "common.cuh"

namespace coarse {
namespace {

constexpr size_t kMaxUnknowns = size_t(1) << 17;  // V*n handled by the static scratch
constexpr size_t kMaxSites = kMaxUnknowns / 16;   // n >= 16
constexpr size_t kPullPushBytes = 5 * kMaxUnknowns * sizeof(double2);
constexpr size_t kCounterBytes = ((kMaxSites + 4) * sizeof(int) + 255) / 256 * 256;
constexpr size_t kPartialDoubles = 2 * 304;
constexpr size_t kScratchBytes = kPullPushBytes + kCounterBytes + kPartialDoubles * sizeof(double) + 256;

// Shared by every call on this device: stencil pull partials and pushes, arrival counters
// (+ error flag), reduction partials, two norms, the reduction counter and {-1, +1}.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Offsets inside g_scratch of the pieces after the pull / push region.
constexpr size_t kOffCnt = kPullPushBytes;
constexpr size_t kOffPartial = kPullPushBytes + kCounterBytes;
constexpr size_t kOffNorms = kOffPartial + kPartialDoubles * sizeof(double);  // 2 doubles
constexpr size_t kOffCounter = kOffNorms + 2 * sizeof(double);                // reduction counter
constexpr size_t kOffCoef = kOffNorms + 4 * sizeof(double);                   // {-1, +1}
static_assert(kOffCoef + 2 * sizeof(double2) <= kScratchBytes, "scratch layout");

// Device address of g_scratch on the current device, looked up once per device; the same
// one-time set-up writes the constant coefficients {-1, +1} of r = -D x + b (a synchronous
// copy, so the first call on a device must not be made while a stream is being captured).
int scratch_address(void** out) {
  int dev = 0;
  COARSE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("coarse_residual_noalloc: device index %d out of range", dev);
    return COARSE_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    COARSE_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    const double2 cst[2] = {make_double2(-1.0, 0.0), make_double2(1.0, 0.0)};
    COARSE_CUDA(cudaMemcpy(static_cast<unsigned char*>(p) + kOffCoef, cst, sizeof(cst), cudaMemcpyHostToDevice));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return COARSE_OK;
}

}  // namespace
}  // namespace coarse

using namespace coarse;

extern "C" int coarse_residual_noalloc(const coarse_op* op, const void* b, const void* x, void* r,
                                       double* norms_host, void* stream) {
  if (!op || !b || !x || !r || !norms_host) {
    set_error("coarse_residual_noalloc: NULL argument");
    return COARSE_ERR_INVALID_ARG;
  }
  if (r == x || r == b) {
    set_error("coarse_residual_noalloc: r must not alias b or x");
    return COARSE_ERR_INVALID_ARG;
  }
  const size_t N = (size_t)op->V * op->n;
  if (N > kMaxUnknowns) {
    set_error("coarse_residual_noalloc: %zu unknowns exceed the static scratch maximum of %zu (V*n)", N,
              kMaxUnknowns);
    return COARSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the call reads its result back and synchronises: it cannot be part of a captured graph
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  COARSE_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    set_error("coarse_residual_noalloc: the stream is being captured (the call synchronises it)");
    return COARSE_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != COARSE_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  int* cnt = reinterpret_cast<int*>(p + kOffCnt);
  double* partial = reinterpret_cast<double*>(p + kOffPartial);
  double* norms = reinterpret_cast<double*>(p + kOffNorms);
  unsigned* counter = reinterpret_cast<unsigned*>(p + kOffCounter);
  const double2* coef = reinterpret_cast<const double2*>(p + kOffCoef);
  // what must start at zero: the stencil's arrival counters and error flag, the reduction counter
  COARSE_CUDA(cudaMemsetAsync(cnt, 0, (op->V + 4) * sizeof(int), s));
  COARSE_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  ApplyArgs a = make_apply_args(op, COARSE_PREC_FP64, x, r);
  a.z = b;
  a.coef = coef;
  a.mode = APPLY_AXPBY;
  a.part = p;
  a.push = p + N * sizeof(double2);
  a.cnt = cnt;
  a.err = cnt + op->V;
  rc = launch_apply(COARSE_PREC_FP64, op->n, a, s);
  if (rc != COARSE_OK) return rc;
  rc = launch_norm2(1, r, (int)N, norms, partial, counter, s);
  if (rc != COARSE_OK) return rc;
  rc = launch_norm2(1, b, (int)N, norms + 1, partial, counter, s);
  if (rc != COARSE_OK) return rc;
  double h[2];
  int err = 0;
  COARSE_CUDA(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  norms_host[0] = sqrt(h[0]);
  norms_host[1] = sqrt(h[1]);
  if (err != 0) {
    // a staged stencil kernel's bounded wait ran out: r is incomplete
    set_error("coarse_residual_noalloc: a bounded wait of the stencil kernel ran out; r is invalid");
    return COARSE_ERR_TIMEOUT;
  }
  return COARSE_OK;
}
