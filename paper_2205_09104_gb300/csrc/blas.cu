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
#include "batch.cuh"

namespace coarse {
namespace {

constexpr int kThreads = 256;
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

// Chunked layout of the Gram-Schmidt kernels: CTA = kW warps, warp chunk = 32*E contiguous
// elements, lane owns elements chunk + lane + 32*e (coalesced for every e).  The w slice
// stays in registers while the kernel sweeps all basis vectors.
constexpr int kW = 8;
constexpr int kMaxQ = 104;  // largest nq + 1 handled in one launch
static_assert(kMaxQ == kBatchMaxQ, "batched reductions size their partials with kBatchMaxQ");

template <class C> __device__ __forceinline__ float2 to_f2(C v) { return make_float2(float(v.x), float(v.y)); }

// per-vector warp reduction of a complex FP32 partial -> FP64 in smem slot
__device__ __forceinline__ void warp_to_smem(float2 acc, double2* slot, int lane) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) *slot = make_double2(double(acc.x), double(acc.y));
}

// dots of the chunk: wp[warp][i] = sum conj(q_i) w  (i < nq), wp[warp][nq] = ||w||^2
template <class C, int E>
__device__ __forceinline__ void chunk_dots(const C* const* q, int nq, const C (&wv)[E], long long base, int N,
                                           int lane, double2* wp) {
  int i = 0;
  for (; i + 2 <= nq; i += 2) {
    const C* q0 = q[i];
    const C* q1 = q[i + 1];
    C a0[E], a1[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) { a0[e] = q0[idx]; a1[e] = q1[idx]; } else { a0[e].x = a0[e].y = 0; a1[e].x = a1[e].y = 0; }
    }
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      cfma_conj(s0, to_f2(a0[e]), to_f2(wv[e]));
      cfma_conj(s1, to_f2(a1[e]), to_f2(wv[e]));
    }
    warp_to_smem(s0, wp + i, lane);
    warp_to_smem(s1, wp + i + 1, lane);
  }
  for (; i < nq; ++i) {
    const C* q0 = q[i];
    float2 s0 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) cfma_conj(s0, to_f2(q0[idx]), to_f2(wv[e]));
    }
    warp_to_smem(s0, wp + i, lane);
  }
  float nn = 0.f;
#pragma unroll
  for (int e = 0; e < E; ++e) nn += float(wv[e].x) * float(wv[e].x) + float(wv[e].y) * float(wv[e].y);
  warp_to_smem(make_float2(nn, 0.f), wp + nq, lane);
}

// FP64 vectors: same, accumulated in FP64 (the FP64 solver path)
template <int E>
__device__ __forceinline__ void chunk_dots(const double2* const* q, int nq, const double2 (&wv)[E], long long base,
                                           int N, int lane, double2* wp) {
  for (int i = 0; i < nq; ++i) {
    const double2* q0 = q[i];
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) cfma_conj(s, q0[idx], wv[e]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (lane == 0) wp[i] = s;
  }
  double nn = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) nn += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
  if (lane == 0) wp[nq] = make_double2(nn, 0.0);
}

// CTA partials (sum over warps in FP64) to the global partial array, then the last CTA reduces.
__device__ void cta_finish(const double2* wp /*[kW][kMaxQ]*/, int nout, double* partial, unsigned* counter,
                           double2* out, double* wnorm2, int norm_slot, int cta = -1, int nch = -1) {
  __syncthreads();
  if (cta < 0) { cta = blockIdx.x; nch = gridDim.x; }
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int w = 0; w < kW; ++w) { re += wp[w * kMaxQ + o].x; im += wp[w * kMaxQ + o].y; }
    partial[(size_t)(2 * o) * nch + cta] = re;
    partial[(size_t)(2 * o + 1) * nch + cta] = im;
  }
  if (last_block(counter, nch)) {
    finish(partial, nout, nch, out, wnorm2, norm_slot);
    if (threadIdx.x == 0) *counter = 0;
  }
}

// h_i = <q_i, w> for i < nq and ||w||^2.
template <class C, int E>
__global__ void __launch_bounds__(32 * kW) k_multidot(const C* const* q, int nq, const C* w, int N, double2* out,
                                                      double* wnorm2, double* partial, unsigned* counter,
                                                      const int* stop) {
  if (stop != nullptr && *stop) return;
  __shared__ double2 wp[kW * kMaxQ];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = ((long long)blockIdx.x * kW + warp) * 32 * E;
  C wv[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const long long idx = base + lane + 32 * e;
    if (idx < N) wv[e] = w[idx]; else { wv[e].x = 0; wv[e].y = 0; }
  }
  chunk_dots(q, nq, wv, base, N, lane, wp + warp * kMaxQ);
  cta_finish(wp, nq + 1, partial, counter, out, wnorm2, nq);
}

// w -= sum_i q_i h_i (negate) or += ; then, if with_dots, out = Q^H w and ||w||^2 of the result,
// else if with_norm only ||w||^2.  One pass over w and two (L2-resident) sweeps of Q's chunk.
template <class C, int E>
__global__ void __launch_bounds__(32 * kW) k_update(const C* const* q, int nq, const double2* h, int negate, C* w,
                                                    int N, int mode /*0: none, 1: norm, 2: dots+norm*/,
                                                    double2* out, double* wnorm2, double* partial,
                                                    unsigned* counter, const int* stop) {
  if (stop != nullptr && *stop) return;
  using T = typename Acc<C>::T;
  __shared__ double2 wp[kW * kMaxQ];
  __shared__ C hc[kMaxQ];
  for (int i = threadIdx.x; i < nq; i += blockDim.x) {
    const double2 v = h[i];
    const double sg = negate ? -1.0 : 1.0;
    hc[i].x = T(sg * v.x);
    hc[i].y = T(sg * v.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = ((long long)blockIdx.x * kW + warp) * 32 * E;
  C wv[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const long long idx = base + lane + 32 * e;
    if (idx < N) wv[e] = w[idx]; else { wv[e].x = 0; wv[e].y = 0; }
  }
  int i = 0;
  for (; i + 4 <= nq; i += 4) {
    const C *q0 = q[i], *q1 = q[i + 1], *q2 = q[i + 2], *q3 = q[i + 3];
    const C h0 = hc[i], h1 = hc[i + 1], h2 = hc[i + 2], h3 = hc[i + 3];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) {
        const C a0 = q0[idx], a1 = q1[idx], a2 = q2[idx], a3 = q3[idx];
        cfma(wv[e], a0, h0); cfma(wv[e], a1, h1); cfma(wv[e], a2, h2); cfma(wv[e], a3, h3);
      }
    }
  }
  for (; i < nq; ++i) {
    const C* q0 = q[i];
    const C h0 = hc[i];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) cfma(wv[e], q0[idx], h0);
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const long long idx = base + lane + 32 * e;
    if (idx < N) w[idx] = wv[e];
  }
  if (mode == 0) return;
  if (mode == 2) {
    chunk_dots(q, nq, wv, base, N, lane, wp + warp * kMaxQ);
    cta_finish(wp, nq + 1, partial, counter, out, wnorm2, nq);
  } else {
    chunk_dots(q, 0, wv, base, N, lane, wp + warp * kMaxQ);
    cta_finish(wp, 1, partial, counter, nullptr, wnorm2, 0);
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

// ------------------------------------------------------------------------------------------
// Batched chunked vector phases: CTA c of the flat grid belongs to the solve found through
// the chunk prefix sums and works on its chunk (c - chunk_off[solve]) of that solve's
// vectors; reductions finish per solve (the solve's own counter and partials).
template <int E>
__global__ void __launch_bounds__(32 * kW) kb_vec(int op, const BSolve* S, int nsolves, const int* chunk_off,
                                                 const int* step_ptr) {
  __shared__ double2 wp[kW * kMaxQ];
  __shared__ float2 hc[kMaxQ];
  const int k = find_solve(chunk_off, nsolves, blockIdx.x);
  const BSolve& s = S[k];
  const int cta = blockIdx.x - chunk_off[k];
  const int step = *step_ptr;
  bool run;
  switch (op) {
    case BV_CGS_DOT: case BV_CGS_UPDDOT: case BV_CGS_UPDNORM: run = bgate(s, BG_STEP); break;
    case BV_PROJ_DOT: case BV_PROJ_UPD: run = bgate(s, BG_ACTIVE) && s.kc > 0; break;
    case BV_RES_UPD: run = bgate(s, BG_TAIL); break;
    default: run = bgate(s, BG_ACTIVE); break;
  }
  if (!run) return;  // uniform over the solve's CTAs
  const float2* const* q = (const float2* const*)(s.kc > 0 ? s.qt : s.vt);
  float2* w = nullptr;
  int nq = 0, upd = 0, dots = 0, norm = 0;
  const double2* h = nullptr;
  double2* out = nullptr;
  double* nout = nullptr;
  switch (op) {
    case BV_CGS_DOT: w = (float2*)s.vt[step + 1]; nq = s.kc + step + 1; dots = 1; out = s.h1; break;
    case BV_CGS_UPDDOT: w = (float2*)s.vt[step + 1]; nq = s.kc + step + 1; upd = 1; h = s.h1; dots = 1; out = s.h2; break;
    case BV_CGS_UPDNORM: w = (float2*)s.vt[step + 1]; nq = s.kc + step + 1; upd = 1; h = s.h2; norm = 1;
      nout = &s.st->wnorm2; break;
    case BV_PROJ_DOT: q = (const float2* const*)s.qt; w = (float2*)s.r; nq = s.kc; dots = 1; out = s.dn.ycoef; break;
    case BV_PROJ_UPD: q = (const float2* const*)s.qt; w = (float2*)s.r; nq = s.kc; upd = 1; h = s.dn.ycoef; norm = 1;
      nout = s.norm2; break;
    case BV_RES_UPD: q = (const float2* const*)s.vt; w = (float2*)s.r; nq = s.st->j + 1; upd = 1; h = s.dn.z; norm = 1;
      nout = s.norm2; break;
    default: w = (float2*)s.r; nq = 0; norm = 1; nout = s.norm2; break;
  }
  const int N = s.N;
  if (upd) {
    for (int i = threadIdx.x; i < nq; i += blockDim.x) hc[i] = make_float2(float(-h[i].x), float(-h[i].y));
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = ((long long)cta * kW + warp) * 32 * E;
  float2 wv[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const long long idx = base + lane + 32 * e;
    wv[e] = idx < N ? w[idx] : make_float2(0.f, 0.f);
  }
  if (upd) {
    for (int i = 0; i < nq; ++i) {
      const float2* qi = q[i];
      const float2 hi = hc[i];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const long long idx = base + lane + 32 * e;
        if (idx < N) cfma(wv[e], qi[idx], hi);
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long idx = base + lane + 32 * e;
      if (idx < N) w[idx] = wv[e];
    }
  }
  if (dots) {
    chunk_dots(q, nq, wv, base, N, lane, wp + warp * kMaxQ);
    cta_finish(wp, nq + 1, s.partial, s.counter, out, nullptr, nq, cta, s.nch);
  } else if (norm) {
    chunk_dots(q, 0, wv, base, N, lane, wp + warp * kMaxQ);
    cta_finish(wp, 1, s.partial, s.counter, nullptr, nout, 0, cta, s.nch);
  }
}

// Batched elementwise phases (same chunk mapping).
template <int E>
__global__ void __launch_bounds__(32 * kW) kb_elem(int op, const BSolve* S, int nsolves, const int* chunk_off,
                                                  const int* step_ptr, int aux, int gate) {
  __shared__ float2 cf[kMaxQ];
  const int k = find_solve(chunk_off, nsolves, blockIdx.x);
  const BSolve& s = S[k];
  const int cta = blockIdx.x - chunk_off[k];
  const int step = *step_ptr;
  bool run = true;
  switch (op) {
    case BE_NORMALIZE: run = s.st->j == step + 1; break;
    case BE_START: run = bgate(s, BG_STEP); break;
    case BE_COMBINE_T: run = bgate(s, BG_TAIL); break;
    case BE_COMBINE_U: run = bgate(s, BG_ACTIVE) && s.kc > 0; break;
    case BE_AXPY_E: run = bgate(s, gate); break;
    case BE_AXPY_E_PROJ: run = bgate(s, BG_ACTIVE) && s.kc > 0; break;
    case BE_TO_LOW: case BE_ADD_LOW: case BE_TO_LOW_F: case BE_EO_SPLIT: case BE_EO_MERGE: case BE_ADD_LOW_F:
      run = bgate(s, BG_NOTDONE);
      break;
    default: run = true; break;
  }
  if (!run) return;
  const int N = belem_full(op) ? s.Nf : s.N;
  int nin = 0;
  const float2* const* in = nullptr;
  if (op == BE_COMBINE_T || op == BE_COMBINE_U) {
    nin = op == BE_COMBINE_T ? s.kc + s.st->j : s.kc;
    in = (const float2* const*)(s.kc > 0 ? s.ut : s.vt);
    for (int i = threadIdx.x; i < nin; i += blockDim.x)
      cf[i] = make_float2(float(s.dn.ycoef[i].x), float(s.dn.ycoef[i].y));
    __syncthreads();
  }
  const double inv_h = s.st->inv_h;
  const double rn = sqrt(fmax(s.norm2[1], 0.0));
  const long long cbase = (long long)cta * kW * 32 * E;
  for (long long idx = cbase + threadIdx.x; idx < cbase + (long long)kW * 32 * E && idx < N; idx += blockDim.x) {
    switch (op) {
      case BE_NORMALIZE: {
        float2* v = (float2*)s.vt[step + 1];
        const float2 a = v[idx];
        v[idx] = make_float2(float(a.x * inv_h), float(a.y * inv_h));
      } break;
      case BE_START: {
        const float2 a = ((const float2*)s.r)[idx];
        ((float2*)s.vt[0])[idx] = make_float2(float(a.x * inv_h), float(a.y * inv_h));
      } break;
      case BE_COMBINE_T:
      case BE_COMBINE_U: {
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < nin; ++i) cfma(acc, in[i][idx], cf[i]);
        ((float2*)s.t)[idx] = acc;
      } break;
      case BE_AXPY_E:
      case BE_AXPY_E_PROJ: {
        const float2 a = ((const float2*)(aux == BS_T ? s.t : s.acc))[idx];
        float2* ev = (float2*)s.e;
        const float2 b = ev[idx];
        ev[idx] = make_float2(b.x + a.x, b.y + a.y);
      } break;
      case BE_TO_LOW: {
        const double2 a = s.r64[idx];
        const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
        ((float2*)s.r)[idx] = make_float2(float(a.x * inv), float(a.y * inv));
        ((float2*)s.e)[idx] = make_float2(0.f, 0.f);
      } break;
      case BE_ADD_LOW:
      case BE_ADD_LOW_F: {
        const float2 d = ((const float2*)(op == BE_ADD_LOW ? s.e : s.f32))[idx];
        double2 x = s.x64[idx];
        x.x = fma(rn, double(d.x), x.x);
        x.y = fma(rn, double(d.y), x.y);
        s.x64[idx] = x;
      } break;
      case BE_TO_LOW_F: {
        const double2 a = s.r64[idx];
        const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
        ((float2*)s.f32)[idx] = make_float2(float(a.x * inv), float(a.y * inv));
      } break;
      case BE_EO_SPLIT: {
        // idx runs over the half vectors: site k of each parity, component c
        const int k = (int)(idx / s.n), c = (int)(idx % s.n);
        const float2* f = (const float2*)s.f32;
        ((float2*)s.re)[idx] = f[(size_t)s.eo_sites[k] * s.n + c];
        ((float2*)s.ro)[idx] = f[(size_t)s.eo_sites[s.V / 2 + k] * s.n + c];
        ((float2*)s.e)[idx] = make_float2(0.f, 0.f);
      } break;
      case BE_EO_MERGE: {
        const int k = (int)(idx / s.n), c = (int)(idx % s.n);
        float2* f = (float2*)s.f32;
        f[(size_t)s.eo_sites[k] * s.n + c] = ((const float2*)s.e)[idx];
        f[(size_t)s.eo_sites[s.V / 2 + k] * s.n + c] = ((const float2*)s.eoe)[idx];
      } break;
      default: s.x64[idx] = make_double2(0.0, 0.0); break;
    }
  }
}

// ||r64||^2 (and ||b64||^2) of every not-yet-converged solve.
template <int E>
__global__ void __launch_bounds__(32 * kW) kb_norm64(const BSolve* S, int nsolves, const int* chunk_off, int which) {
  __shared__ double2 wp[kW * kMaxQ];
  const int k = find_solve(chunk_off, nsolves, blockIdx.x);
  const BSolve& s = S[k];
  if (!bgate(s, BG_NOTDONE)) return;
  const int cta = blockIdx.x - chunk_off[k];
  const double2* v = which == 1 ? s.r64 : s.b64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = ((long long)cta * kW + warp) * 32 * E;
  double nn = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const long long idx = base + lane + 32 * e;
    if (idx < s.Nf) { const double2 a = v[idx]; nn += a.x * a.x + a.y * a.y; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
  if (lane == 0) wp[warp * kMaxQ] = make_double2(nn, 0.0);
  cta_finish(wp, 1, s.partial, s.counter, nullptr, s.norm2 + which, 0, cta, s.nchf);
}

}  // namespace

namespace {
int chunk_elems(int N) { return N <= (1 << 18) ? 4 : (N <= (1 << 20) ? 8 : 16); }
int chunk_grid(int N, int E) { return (int)(((long long)N + 32LL * kW * E - 1) / (32LL * kW * E)); }

template <class C>
int multidot_t(const void* const* q, int nq, const void* w, int N, double2* out, double* wnorm2, double* partial,
               unsigned* counter, const int* stop, cudaStream_t s) {
  const int E = chunk_elems(N);
  const int grid = chunk_grid(N, E);
  auto qq = (const C* const*)q;
  auto ww = (const C*)w;
  if (E == 4) k_multidot<C, 4><<<grid, 32 * kW, 0, s>>>(qq, nq, ww, N, out, wnorm2, partial, counter, stop);
  else if (E == 8) k_multidot<C, 8><<<grid, 32 * kW, 0, s>>>(qq, nq, ww, N, out, wnorm2, partial, counter, stop);
  else k_multidot<C, 16><<<grid, 32 * kW, 0, s>>>(qq, nq, ww, N, out, wnorm2, partial, counter, stop);
  return grid;
}

template <class C>
int update_t(const void* const* q, int nq, const double2* h, int negate, void* w, int N, int mode, double2* out,
             double* wnorm2, double* partial, unsigned* counter, const int* stop, cudaStream_t s) {
  const int E = chunk_elems(N);
  const int grid = chunk_grid(N, E);
  auto qq = (const C* const*)q;
  auto ww = (C*)w;
  if (E == 4)
    k_update<C, 4><<<grid, 32 * kW, 0, s>>>(qq, nq, h, negate, ww, N, mode, out, wnorm2, partial, counter, stop);
  else if (E == 8)
    k_update<C, 8><<<grid, 32 * kW, 0, s>>>(qq, nq, h, negate, ww, N, mode, out, wnorm2, partial, counter, stop);
  else
    k_update<C, 16><<<grid, 32 * kW, 0, s>>>(qq, nq, h, negate, ww, N, mode, out, wnorm2, partial, counter, stop);
  return grid;
}
}  // namespace

int max_reduction_chunks(int N) { return chunk_grid(N, chunk_elems(N)); }

int launch_multidot(int prec64, const void* const* q, int nq, const void* w, int N, double2* out, double* wnorm2,
                    double* partial, unsigned* counter, const int* stop, cudaStream_t s) {
  if (nq + 1 > kMaxQ) { set_error("multi-dot of %d vectors exceeds %d", nq, kMaxQ - 1); return COARSE_ERR_INVALID_ARG; }
  if (prec64) multidot_t<double2>(q, nq, w, N, out, wnorm2, partial, counter, stop, s);
  else multidot_t<float2>(q, nq, w, N, out, wnorm2, partial, counter, stop, s);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_update(int prec64, const void* const* q, int nq, const double2* h, int negate, void* w, int N,
                  int mode, double2* out_dots, double* wnorm2, double* partial, unsigned* counter,
                  const int* stop, cudaStream_t s) {
  if (nq + 1 > kMaxQ) { set_error("update with %d vectors exceeds %d", nq, kMaxQ - 1); return COARSE_ERR_INVALID_ARG; }
  if (prec64) update_t<double2>(q, nq, h, negate, w, N, mode, out_dots, wnorm2, partial, counter, stop, s);
  else update_t<float2>(q, nq, h, negate, w, N, mode, out_dots, wnorm2, partial, counter, stop, s);
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

namespace coarse {

int launch_bvec(int op, const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E, const int* step,
                cudaStream_t s) {
  if (total_chunks <= 0) return COARSE_OK;
  if (E == 4) kb_vec<4><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step);
  else if (E == 8) kb_vec<8><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step);
  else kb_vec<16><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_belem(int op, const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E, const int* step,
                 int aux, int gate, cudaStream_t s) {
  if (total_chunks <= 0) return COARSE_OK;
  if (E == 4) kb_elem<4><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step, aux, gate);
  else if (E == 8) kb_elem<8><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step, aux, gate);
  else kb_elem<16><<<total_chunks, 32 * kW, 0, s>>>(op, S, nsolves, chunk_off, step, aux, gate);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_bnorms64(const BSolve* S, int nsolves, const int* chunk_off, int total_chunks, int E, int which,
                    cudaStream_t s) {
  if (total_chunks <= 0) return COARSE_OK;
  if (E == 4) kb_norm64<4><<<total_chunks, 32 * kW, 0, s>>>(S, nsolves, chunk_off, which);
  else if (E == 8) kb_norm64<8><<<total_chunks, 32 * kW, 0, s>>>(S, nsolves, chunk_off, which);
  else kb_norm64<16><<<total_chunks, 32 * kW, 0, s>>>(S, nsolves, chunk_off, which);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int batch_chunk_elems(int maxN) { return chunk_elems(maxN); }
int batch_chunks(int N, int E) { return chunk_grid(N, E); }

}  // namespace coarse
