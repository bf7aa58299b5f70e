// Vector kernels of the Krylov solver: fused Gram-Schmidt dots and updates
// (Sec. 3.1: classical Gram-Schmidt fuses the j inner products of Arnoldi
// step j into one reduction; Sec. 3.4 merges the deflation dots with C_k into
// the same reduction), linear combinations of basis vectors, conversions.
//
// Reductions: every thread accumulates in the vector precision, the block
// reduces in FP64, per-block partials go to a scratch array and the last
// block to finish (global counter) sums them in a fixed order, so results are
// deterministic and no second launch is needed.
#include "common.cuh"
#include "solver_state.cuh"

namespace coarse {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;     // vectors per CTA row of the multi-dot
constexpr int kMaxChunks = 304;

template <class C> struct Acc;
template <> struct Acc<float2> { using T = float; };
template <> struct Acc<double2> { using T = double; };

int chunks_for(int N) {
  int c = (N + kThreads * 4 - 1) / (kThreads * 4);
  if (c > kMaxChunks) c = kMaxChunks;
  return c < 1 ? 1 : c;
}

// Block-wide FP64 sum of kv values per thread (in place into s[kv] of thread 0's view).
template <int KV>
__device__ void block_sum(double (&v)[KV], double* sh /* [kThreads/32][KV] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KV; ++i)
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < KV; ++i) sh[warp * KV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      double s = lane < kThreads / 32 ? sh[lane * KV + i] : 0.0;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      v[i] = s;
    }
  }
  __syncthreads();
}

// Last block: out[o] = sum_c partial[o][c] for o < nout (partial as double pairs).
__device__ void finish(const double* partial, int nout, int nch, double2* out, double* wnorm2, int norm_slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = warp; o < nout; o += kThreads / 32) {
    double re = 0.0, im = 0.0;
    for (int c = lane; c < nch; c += 32) {
      re += partial[(size_t)(2 * o) * nch + c];
      im += partial[(size_t)(2 * o + 1) * nch + c];
    }
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) {
      if (o == norm_slot) {
        if (wnorm2) *wnorm2 = re;
      } else if (out) {
        out[o] = make_double2(re, im);
      }
    }
  }
}

__device__ bool last_block(unsigned* counter, unsigned total) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == total - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// h_i = <q_i, w> for i < nq and ||w||^2 (slot nq).  grid = (chunks, ceil((nq+1)/kGroup)).
template <class C>
__global__ void __launch_bounds__(kThreads) k_multidot(const C* const* q, int nq, const C* w, int N, double2* out,
                                                       double* wnorm2, double* partial, unsigned* counter,
                                                       const int* stop) {
  if (stop != nullptr && *stop) return;
  using T = typename Acc<C>::T;
  __shared__ double sh[kThreads / 32 * 2 * kGroup];
  const int nch = gridDim.x;
  const int g0 = blockIdx.y * kGroup;
  T re[kGroup], im[kGroup];
#pragma unroll
  for (int i = 0; i < kGroup; ++i) { re[i] = 0; im[i] = 0; }
  const C* qp[kGroup];
#pragma unroll
  for (int i = 0; i < kGroup; ++i) qp[i] = (g0 + i < nq) ? q[g0 + i] : nullptr;
  const int stride = nch * kThreads;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < N; e += stride) {
    const C wv = w[e];
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
      const int idx = g0 + i;
      if (idx < nq) {
        const C a = qp[i][e];
        re[i] = fma(a.x, wv.x, re[i]); re[i] = fma(a.y, wv.y, re[i]);
        im[i] = fma(a.x, wv.y, im[i]); im[i] = fma(-a.y, wv.x, im[i]);
      } else if (idx == nq) {
        re[i] = fma(wv.x, wv.x, re[i]); re[i] = fma(wv.y, wv.y, re[i]);
      }
    }
  }
  double v[2 * kGroup];
#pragma unroll
  for (int i = 0; i < kGroup; ++i) { v[2 * i] = re[i]; v[2 * i + 1] = im[i]; }
  block_sum<2 * kGroup>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
      const int o = g0 + i;
      if (o <= nq) {
        partial[(size_t)(2 * o) * nch + blockIdx.x] = v[2 * i];
        partial[(size_t)(2 * o + 1) * nch + blockIdx.x] = v[2 * i + 1];
      }
    }
  }
  if (last_block(counter, gridDim.x * gridDim.y)) {
    finish(partial, nq + 1, nch, out, wnorm2, nq);
    if (threadIdx.x == 0) *counter = 0;
  }
}

// w = w -/+ sum_i q_i h_i ; optionally ||w||^2 of the result.
template <class C>
__global__ void __launch_bounds__(kThreads) k_update(const C* const* q, int nq, const double2* h, int negate, C* w,
                                                     int N, int with_norm, double* wnorm2, double* partial,
                                                     unsigned* counter, const int* stop) {
  if (stop != nullptr && *stop) return;
  using T = typename Acc<C>::T;
  extern __shared__ unsigned char smem_raw[];
  C* hc = reinterpret_cast<C*>(smem_raw);
  const C** qs = reinterpret_cast<const C**>(smem_raw + sizeof(C) * nq + (16 - (sizeof(C) * nq) % 16) % 16);
  __shared__ double sh[kThreads / 32 * 2];
  for (int i = threadIdx.x; i < nq; i += kThreads) {
    const double2 v = h[i];
    const double sg = negate ? -1.0 : 1.0;
    hc[i].x = T(sg * v.x);
    hc[i].y = T(sg * v.y);
    qs[i] = q[i];
  }
  __syncthreads();
  T nrm = 0;
  const int stride = gridDim.x * kThreads;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < N; e += stride) {
    C acc = w[e];
    int i = 0;
    for (; i + 4 <= nq; i += 4) {
      const C a0 = qs[i][e], a1 = qs[i + 1][e], a2 = qs[i + 2][e], a3 = qs[i + 3][e];
      cfma(acc, a0, hc[i]); cfma(acc, a1, hc[i + 1]); cfma(acc, a2, hc[i + 2]); cfma(acc, a3, hc[i + 3]);
    }
    for (; i < nq; ++i) cfma(acc, qs[i][e], hc[i]);
    w[e] = acc;
    nrm = fma(acc.x, acc.x, nrm);
    nrm = fma(acc.y, acc.y, nrm);
  }
  if (!with_norm) return;
  double v[2] = {double(nrm), 0.0};
  block_sum<2>(v, sh);
  const int nch = gridDim.x;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = v[0];
    partial[nch + blockIdx.x] = 0.0;
  }
  if (last_block(counter, gridDim.x)) {
    finish(partial, 1, nch, nullptr, wnorm2, 0);
    if (threadIdx.x == 0) *counter = 0;
  }
}

// out_i (+)= sum_j in_j coef[j*ldc + i], i < nout, tile of TILE outputs per pass.
template <class C, int TILE>
__global__ void __launch_bounds__(kThreads) k_combine(const C* const* in, int nin, const double2* coef, int ldc,
                                                      C* const* out, int nout, int accumulate, int N, const int* stop) {
  if (stop != nullptr && *stop) return;
  using T = typename Acc<C>::T;
  extern __shared__ unsigned char smem_raw[];
  C* cf = reinterpret_cast<C*>(smem_raw);  // [nin][TILE]
  const int o0 = blockIdx.y * TILE;
  for (int k = threadIdx.x; k < nin * TILE; k += kThreads) {
    const int j = k / TILE, i = k % TILE;
    double2 v = (o0 + i < nout) ? coef[(size_t)j * ldc + o0 + i] : make_double2(0.0, 0.0);
    cf[k].x = T(v.x);
    cf[k].y = T(v.y);
  }
  __syncthreads();
  const int stride = gridDim.x * kThreads;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < N; e += stride) {
    C acc[TILE];
#pragma unroll
    for (int i = 0; i < TILE; ++i) { acc[i].x = 0; acc[i].y = 0; }
    for (int j = 0; j < nin; ++j) {
      const C a = in[j][e];
#pragma unroll
      for (int i = 0; i < TILE; ++i) cfma(acc[i], a, cf[j * TILE + i]);
    }
#pragma unroll
    for (int i = 0; i < TILE; ++i) {
      if (o0 + i < nout) {
        C* o = out[o0 + i];
        if (accumulate) o[e] = cadd(o[e], acc[i]);
        else o[e] = acc[i];
      }
    }
  }
}

// y = alpha * (inv ? *inv : 1) * x; runs only if gate == nullptr or *gate == gate_val.
template <class C>
__global__ void k_scale(const C* x, const double* inv, double2 alpha, C* y, int N, const int* gate, int gate_val) {
  if (gate != nullptr && *gate != gate_val) return;
  using T = typename Acc<C>::T;
  double ar = alpha.x, ai = alpha.y;
  if (inv != nullptr) { const double s = *inv; ar *= s; ai *= s; }
  const C a{T(ar), T(ai)};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) y[e] = cmul(a, x[e]);
}

template <class C>
__global__ void k_axpy(const C* x, C* y, double2 alpha, int N, const int* stop) {
  if (stop != nullptr && *stop) return;
  using T = typename Acc<C>::T;
  const C a{T(alpha.x), T(alpha.y)};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    C v = y[e];
    cfma(v, a, x[e]);
    y[e] = v;
  }
}

template <class C>
__global__ void __launch_bounds__(kThreads) k_norm2(const C* x, int N, double* out, double* partial, unsigned* counter) {
  using T = typename Acc<C>::T;
  __shared__ double sh[kThreads / 32 * 2];
  T s = 0;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < N; e += gridDim.x * kThreads) {
    const C v = x[e];
    s = fma(v.x, v.x, s);
    s = fma(v.y, v.y, s);
  }
  double v[2] = {double(s), 0.0};
  block_sum<2>(v, sh);
  const int nch = gridDim.x;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = v[0];
    partial[nch + blockIdx.x] = 0.0;
  }
  if (last_block(counter, gridDim.x)) {
    finish(partial, 1, nch, nullptr, out, 0);
    if (threadIdx.x == 0) *counter = 0;
  }
}

__global__ void k_to_low(const double2* x, const double* nrm2, float2* y, int N) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const double2 v = x[e];
    y[e] = make_float2(float(v.x * inv), float(v.y * inv));
  }
}

__global__ void k_add_low(double2* x, const double* nrm2, const float2* e32, int N) {
  const double s = sqrt(*nrm2);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const float2 d = e32[e];
    double2 v = x[e];
    v.x = fma(s, double(d.x), v.x);
    v.y = fma(s, double(d.y), v.y);
    x[e] = v;
  }
}

template <class C>
__global__ void k_sigma3(const C* x, C* y, int n, int total) {
  const int nv = n / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    C v = x[e];
    if ((e % n) >= nv) { v.x = -v.x; v.y = -v.y; }
    y[e] = v;
  }
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based hash -> uniform doubles -> Box-Muller.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_fill_gaussian(double2* x, int N, uint64_t seed) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ splitmix64(2ull * (uint64_t)e));
    const uint64_t b = splitmix64(seed ^ splitmix64(2ull * (uint64_t)e + 1ull));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    x[e] = make_double2(rad * cs, rad * sn);
  }
}

template <class C>
__global__ void k_copy_to(const double2* x, C* y, int N) {
  using T = typename Acc<C>::T;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const double2 v = x[e];
    y[e].x = T(v.x);
    y[e].y = T(v.y);
  }
}

template <class C>
__global__ void k_check_finite(const C* x, int N, int* flag) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const C v = x[e];
    if (!isfinite(double(v.x)) || !isfinite(double(v.y))) { *flag = 1; return; }
  }
}

int elem_grid(int N) {
  int g = (N + 255) / 256;
  return g > 152 * 8 ? 152 * 8 : (g < 1 ? 1 : g);
}

}  // namespace

int launch_multidot(int prec64, const void* const* q, int nq, const void* w, int N, double2* out, double* wnorm2,
                    double* partial, unsigned* counter, const int* stop, cudaStream_t s) {
  const dim3 grid(chunks_for(N), (nq + 1 + kGroup - 1) / kGroup);
  if (prec64)
    k_multidot<double2><<<grid, kThreads, 0, s>>>((const double2* const*)q, nq, (const double2*)w, N, out, wnorm2,
                                                  partial, counter, stop);
  else
    k_multidot<float2><<<grid, kThreads, 0, s>>>((const float2* const*)q, nq, (const float2*)w, N, out, wnorm2,
                                                 partial, counter, stop);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_update(int prec64, const void* const* q, int nq, const double2* h, int negate, void* w, int N,
                  int with_dot, double2* /*out_dots*/, double* wnorm2, double* partial, unsigned* counter,
                  const int* stop, cudaStream_t s) {
  const int grid = chunks_for(N);
  const size_t csz = prec64 ? sizeof(double2) : sizeof(float2);
  const size_t smem = csz * nq + 16 + sizeof(void*) * nq;
  if (prec64)
    k_update<double2><<<grid, kThreads, smem, s>>>((const double2* const*)q, nq, h, negate, (double2*)w, N, with_dot,
                                                   wnorm2, partial, counter, stop);
  else
    k_update<float2><<<grid, kThreads, smem, s>>>((const float2* const*)q, nq, h, negate, (float2*)w, N, with_dot,
                                                  wnorm2, partial, counter, stop);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_combine(int prec64, const void* const* in, int nin, const double2* coef, int ldc, void* const* out,
                   int nout, int accumulate, int N, const int* stop, cudaStream_t s) {
  if (nin <= 0 || nout <= 0) return COARSE_OK;
  const int tile = nout == 1 ? 1 : 8;
  const dim3 grid(chunks_for(N), (nout + tile - 1) / tile);
  const size_t csz = prec64 ? sizeof(double2) : sizeof(float2);
  const size_t smem = csz * nin * tile;
  if (prec64) {
    if (tile == 1)
      k_combine<double2, 1><<<grid, kThreads, smem, s>>>((const double2* const*)in, nin, coef, ldc,
                                                         (double2* const*)out, nout, accumulate, N, stop);
    else
      k_combine<double2, 8><<<grid, kThreads, smem, s>>>((const double2* const*)in, nin, coef, ldc,
                                                         (double2* const*)out, nout, accumulate, N, stop);
  } else {
    if (tile == 1)
      k_combine<float2, 1><<<grid, kThreads, smem, s>>>((const float2* const*)in, nin, coef, ldc,
                                                        (float2* const*)out, nout, accumulate, N, stop);
    else
      k_combine<float2, 8><<<grid, kThreads, smem, s>>>((const float2* const*)in, nin, coef, ldc,
                                                        (float2* const*)out, nout, accumulate, N, stop);
  }
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_scale(int prec64, const void* x, const double* inv, double2 alpha, void* y, int N, const int* gate,
                 int gate_val, cudaStream_t s) {
  if (prec64) k_scale<double2><<<elem_grid(N), 256, 0, s>>>((const double2*)x, inv, alpha, (double2*)y, N, gate, gate_val);
  else k_scale<float2><<<elem_grid(N), 256, 0, s>>>((const float2*)x, inv, alpha, (float2*)y, N, gate, gate_val);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_axpy(int prec64, const void* x, void* y, double2 alpha, int N, const int* stop, cudaStream_t s) {
  if (prec64) k_axpy<double2><<<elem_grid(N), 256, 0, s>>>((const double2*)x, (double2*)y, alpha, N, stop);
  else k_axpy<float2><<<elem_grid(N), 256, 0, s>>>((const float2*)x, (float2*)y, alpha, N, stop);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_norm2(int prec64, const void* x, int N, double* out, double* partial, unsigned* counter, cudaStream_t s) {
  const int grid = chunks_for(N);
  if (prec64) k_norm2<double2><<<grid, kThreads, 0, s>>>((const double2*)x, N, out, partial, counter);
  else k_norm2<float2><<<grid, kThreads, 0, s>>>((const float2*)x, N, out, partial, counter);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_to_low(const double2* x64, const double* nrm2, float2* y32, int N, cudaStream_t s) {
  k_to_low<<<elem_grid(N), 256, 0, s>>>(x64, nrm2, y32, N);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_add_low(double2* x64, const double* nrm2, const float2* e32, int N, cudaStream_t s) {
  k_add_low<<<elem_grid(N), 256, 0, s>>>(x64, nrm2, e32, N);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_sigma3(int prec64, const void* x, void* y, int n, int V, cudaStream_t s) {
  const int total = n * V;
  if (prec64) k_sigma3<double2><<<elem_grid(total), 256, 0, s>>>((const double2*)x, (double2*)y, n, total);
  else k_sigma3<float2><<<elem_grid(total), 256, 0, s>>>((const float2*)x, (float2*)y, n, total);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_fill_gaussian(double2* x, int N, uint64_t seed, cudaStream_t s) {
  k_fill_gaussian<<<elem_grid(N), 256, 0, s>>>(x, N, seed);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_copy_to(int prec64, const double2* x64, void* y, int N, cudaStream_t s) {
  if (prec64) k_copy_to<double2><<<elem_grid(N), 256, 0, s>>>(x64, (double2*)y, N);
  else k_copy_to<float2><<<elem_grid(N), 256, 0, s>>>(x64, (float2*)y, N);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_check_finite(int prec64, const void* x, int N, int* flag, cudaStream_t s) {
  if (prec64) k_check_finite<double2><<<elem_grid(N), 256, 0, s>>>((const double2*)x, N, flag);
  else k_check_finite<float2><<<elem_grid(N), 256, 0, s>>>((const float2*)x, N, flag);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace coarse
