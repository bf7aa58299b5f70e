// FP64 FMA throughput of the device, measured with a plain dependent-FMA loop.  The FP64
// stencil (the refinement residual r = b - D_c x) is bound by this rate rather than by HBM on
// GB300, whose FP64 rate is far below its bandwidth-to-flop balance; the measured peak is the
// denominator of that kernel's roofline.
#include <cuda_runtime.h>

#include "common.cuh"

namespace coarse {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread, to cover the pipeline latency

__global__ void __launch_bounds__(256) k_fma_loop(double* sink, int iters, double a, double b) {
  double x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s > 1e300) sink[0] = s;  // never true (every chain stays within [0, 8)); keeps the loop alive
}

}  // namespace
}  // namespace coarse

using namespace coarse;

extern "C" int coarse_measure_fp64_fma(int iters, double* tflops_host, void* stream) {
  if (!tflops_host || iters < 1) {
    set_error("coarse_measure_fp64_fma: need iters >= 1 and an output");
    return COARSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  COARSE_CUDA(cudaGetDevice(&dev));
  COARSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 8 resident CTAs of 256 threads per SM
  cudaEvent_t e0, e1;
  COARSE_CUDA(cudaEventCreate(&e0));
  COARSE_CUDA(cudaEventCreate(&e1));
  // a = 1 - 2^-30, b = 2^-31: the chains stay finite and never reach the sink's test value
  const double a = 1.0 - 9.313225746154785e-10, b = 4.656612873077393e-10;
  k_fma_loop<<<blocks, 256, 0, s>>>(nullptr, iters, a, b);  // warm-up
  note_launch();
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_loop<<<blocks, 256, 0, s>>>(nullptr, iters, a, b);
    note_launch();
    cudaEventRecord(e1, s);
    COARSE_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  COARSE_CUDA(cudaGetLastError());
  const double flops = 2.0 * kChains * (double)iters * blocks * 256.0;
  *tflops_host = flops / (best * 1e-3) / 1e12;
  return COARSE_OK;
}
