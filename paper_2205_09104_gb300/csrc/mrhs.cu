// Multi-right-hand-side apply Y = D_c X on tensor cores (BF16 blocks and vector fragments,
// FP32 accumulation) for one operator, the repacking of its BF16 blocks into the
// fragment-native layout, and the packing of the vectors into BF16 B fragments.  The pipeline
// is mrhs_ring.cuh; the per-block tensor-core products are mrhs_core.cuh.
#include <cstdio>
#include <vector>

#include "mrhs_ring.cuh"
#include "mrhs_tc.cuh"
#include "tune.cuh"

namespace coarse {
namespace {

// BF16 blocks [V][5][n][n] (complex, re in the low half) -> fragment-native planes.
__global__ void k_pack_mrhs(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int V, int n) {
  const int NT = n / 16;
  const size_t total = (size_t)V * 5 * n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int w = (int)(i & 3), l = (int)((i >> 2) & 31);
    size_t rest = i >> 7;
    const int p = (int)(rest & 1);
    rest >>= 1;
    const int tk = (int)(rest % NT);
    rest /= NT;
    const int ti = (int)(rest % NT);
    rest /= NT;  // rest = x * 5 + b
    const int g = l >> 2, t = l & 3;
    const int row = 16 * ti + g + 8 * (w & 1), col = 16 * tk + 2 * t + 8 * (w >> 1);
    const uint32_t* s = src + rest * n * n + (size_t)row * n + col;
    const uint32_t u0 = s[0], u1 = s[1];
    dst[i] = p ? __byte_perm(u0, u1, 0x7632) : __byte_perm(u0, u1, 0x5410);
  }
}

// complex64 columns x + q*ldx (q < R) -> fragment-native BF16 B operands (layout in
// mrhs_core.cuh), zeros for the columns R .. 4T-1 of the last tile.  One thread per site, padded
// column q and entry pair kp (coalesced 16-byte reads along kp); entry pair kp = 8kt + 4w + t
// feeds word w of lane (2(q%4) + part, t) of tile (q/4, kt), the real part to the even lane.
__global__ void k_pack_mrhs_x(const float2* __restrict__ x, long long ldx, int R, int T, int V, int n,
                              uint32_t* __restrict__ xb) {
  const int NT = n / 16, HP = n / 2;  // entry pairs per vector
  const size_t total = (size_t)V * (kMrhsTile * T) * HP;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kp = (int)(i % HP);
    const size_t rest = i / HP;
    const int q = (int)(rest % (kMrhsTile * T));
    const size_t site = rest / (kMrhsTile * T);
    uint32_t re = 0u, im = 0u;
    if (q < R) {
      const float4 e = __ldg(reinterpret_cast<const float4*>(x + q * ldx + site * n + 2 * kp));
      re = bf2_bits(e.x, e.z);
      im = bf2_bits(e.y, e.w);
    }
    const int kt = kp >> 3, w = (kp >> 2) & 1, t = kp & 3, tl = q / kMrhsTile, g = 2 * (q % kMrhsTile);
    uint32_t* dst = xb + ((site * T + tl) * NT + kt) * 64 + (4 * g + t) * 2 + w;
    dst[0] = re;
    dst[8] = im;  // lane + 4 (g + 1)
  }
}

struct MrhsArgs {
  const uint4* frag;  // fragment-native BF16 blocks
  const int* nb;      // [V][8]
  const float2* x;    // column q at x + q * ldx (complex64, [V][n]; read by the twisted-mass term)
  const uint2* xb;    // the same columns as BF16 B fragments, [V][T][NT][32] uint2
  float2* y;
  long long ldx, ldy;
  int R;              // columns of this pass (1 .. 12)
  int V;
  int S;              // stages
  uint32_t SB;        // bytes per stage
  float mu;           // signed twisted mass (-mu for the adjoint)
  int adj;
  int* err;
  const void* tcblk;  // the blocks as tcgen05 core-matrix planes (null: the tcgen05 kernel is not offered)
};

template <int N, int P> struct MrhsShape {
  static constexpr int NT = N / 16;
  static constexpr int WC = P * NT;            // consumer warps
  static constexpr int THREADS = (WC + 1) * 32;
};

// One operator, columns x + q*ldx, plain or adjoint product (a: the kernel's __grid_constant__
// parameter, read through the constant bank rather than copied into registers).
template <int N, int T>
struct MrhsPlain {
  static constexpr bool kRuntimeT = false;
  const MrhsArgs* pa;
  __device__ int ngroups(int P) const { return (pa->V + P - 1) / P; }
  __device__ MrhsGroup group(int g, int P) const {
    const MrhsArgs& a = *pa;
    MrhsGroup r;
    r.frag = a.frag;
    r.nb = a.nb;
    r.xb = a.xb;
    r.V = a.V;
    r.x0 = g * P;
    r.np = a.V - r.x0 < P ? a.V - r.x0 : P;
    r.T = T;
    r.tag = 0;
    return r;
  }
  __device__ int adjoint() const { return pa->adj; }
  __device__ void finish(const MrhsGroup&, int x, int rt, const MrhsAcc<T>& acc) const {
    const MrhsArgs& a = *pa;
    const int lane = threadIdx.x & 31, t = lane & 3, g = lane >> 2;
#pragma unroll
    for (int tl = 0; tl < T; ++tl) {
      const int q = kMrhsTile * tl + t;
      if (q >= a.R) continue;
      float2 y0, y1;
      mrhs_rows_out<N, T>(acc, tl, rt, a.x + q * a.ldx + (size_t)x * N, a.mu, a.adj, y0, y1);
      float2* ys = a.y + q * a.ldy + (size_t)x * N + 16 * rt + g;
      ys[0] = y0;
      ys[8] = y1;
    }
  }
};

template <int N, int T, int P>
__global__ void __launch_bounds__(mrhs_threads(N, P), mrhs_min_blocks(N, P)) k_apply_mrhs(const __grid_constant__ MrhsArgs a) {
  mrhs_ring<N, P, T>(MrhsPlain<N, T>{&a}, a.S, a.SB, a.err);
}

constexpr int kMrhsMaxSmem = 200 * 1024;

// Launch with P sites per stage and S stages (S = 0: as many as fit 64 KB).
template <int N, int T, int P>
int launch_mrhs_cfg(MrhsArgs a, int S, cudaStream_t s) {
  using Sh = MrhsShape<N, P>;
  static bool attr = false;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_apply_mrhs<N, T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMrhsMaxSmem));
    attr = true;
  }
  a.SB = mrhs_stage_bytes(N, P, T);
  if (S <= 0) S = (int)((64u * 1024u) / a.SB);
  S = S < 2 ? 2 : (S > 8 ? 8 : S);
  while (S > 2 && (size_t)S * a.SB + 16 * S > (size_t)kMrhsMaxSmem) --S;
  a.S = S;
  const size_t smem = (size_t)S * a.SB + 2 * S * sizeof(uint64_t);
  if (smem > (size_t)kMrhsMaxSmem) {
    set_error("multi-RHS apply: %zu bytes of shared memory for %d stages", smem, S);
    return COARSE_ERR_INVALID_ARG;
  }
  int per_sm = 0;
  COARSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_mrhs<N, T, P>, Sh::THREADS, smem));
  if (per_sm < 1) {
    set_error("multi-RHS apply: no CTA fits (%zu bytes of shared memory)", smem);
    return COARSE_ERR_INVALID_ARG;
  }
  const int ngroups = (a.V + P - 1) / P;
  int grid = per_sm * sm_count();
  if (grid > ngroups) grid = ngroups;
  k_apply_mrhs<N, T, P><<<grid, Sh::THREADS, smem, s>>>(a);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

// configurations offered to the autotuner: (P, S); the first is the static default
// (P = 100 + k: the tcgen05 kernel with k CTAs per SM and stages S, 0: all that fit)
template <int N, int T>
std::vector<TuneChoice> mrhs_candidates(bool tc) {
  std::vector<TuneChoice> c;
  if constexpr (T > kMrhsMaxT) {  // 16-column passes: the tcgen05 kernel only
    if (tc && (N == 32 || N == 48))
      for (int k = 1; k <= 2; ++k) c.push_back({100 + k, 0, 0});
    return c;
  }
  const int def_p = N == 16 ? 4 : (N == 32 ? 2 : 1);
  const int ps[3] = {N == 16 ? 2 : 1, N == 16 ? 4 : 2, N == 16 ? 8 : 4};
  c.push_back({def_p, 0, 0});
  for (int P : ps) {
    if (P * (N / 16) > 8) continue;
    for (int S : {3, 5, 8})
      if (!(P == def_p && S == 0)) c.push_back({P, S, 0});
  }
  if (tc && (N == 32 || N == 48)) {
    const int max_ctas = T <= 2 ? 3 : 2;  // tensor-memory columns: 128 per CTA for T <= 2, else 256
    for (int k = 1; k <= max_ctas; ++k) c.push_back({100 + k, 0, 0});
  }
  return c;
}

// the columns as mma.sync B fragments (k_pack_mrhs_x), then the mma.sync kernel
template <int N, int T, int P>
int launch_mrhs_frag(const MrhsArgs& a, int S, cudaStream_t s) {
  const size_t total = (size_t)a.V * (kMrhsTile * T) * (N / 2);
  size_t grid = (total + 255) / 256;
  if (grid > (size_t)sm_count() * 16) grid = (size_t)sm_count() * 16;
  k_pack_mrhs_x<<<(int)grid, 256, 0, s>>>(a.x, a.ldx, a.R, T, a.V, N, (uint32_t*)a.xb);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return launch_mrhs_cfg<N, T, P>(a, S, s);
}

template <int N, int T>
int launch_mrhs_choice(const MrhsArgs& a, const TuneChoice& c, cudaStream_t s) {
  switch (c.a) {
    case 1:
      if constexpr (T <= kMrhsMaxT) return launch_mrhs_frag<N, T, 1>(a, c.b, s);
      break;
    case 2:
      if constexpr (T <= kMrhsMaxT) return launch_mrhs_frag<N, T, 2>(a, c.b, s);
      break;
    case 4:
      if constexpr (T <= kMrhsMaxT) return launch_mrhs_frag<N, T, 4>(a, c.b, s);
      break;
    case 8:
      if constexpr (N == 16 && T <= kMrhsMaxT) return launch_mrhs_frag<N, T, 8>(a, c.b, s);
      break;
    case 101:
    case 102:
    case 103:
      if (a.tcblk) {
        TcArgs t{};
        t.blk = static_cast<const unsigned char*>(a.tcblk);
        t.nb = a.nb;
        t.x = a.x;
        t.xv = (unsigned char*)const_cast<uint2*>(a.xb);
        t.y = a.y;
        t.ldx = a.ldx;
        t.ldy = a.ldy;
        t.R = a.R;
        t.V = a.V;
        t.n = N;
        t.mu = a.mu;
        t.adj = a.adj;
        t.err = a.err;
        return launch_apply_mrhs_tc(t, T, c.a - 100, c.b, s);
      }
      break;
  }
  set_error("multi-RHS apply: no configuration with %d sites per stage for n = %d", c.a, N);
  return COARSE_ERR_INVALID_ARG;
}

template <int N, int T>
int launch_mrhs_t(const MrhsArgs& a, cudaStream_t s) {
  char key[96];
  snprintf(key, sizeof(key), "mrhs/n%d/t%d/v%d", N, T, tune_bucket(a.V));
  TuneChoice c;
  int rc = tune_pick(key, mrhs_candidates<N, T>(a.tcblk != nullptr), [&](const TuneChoice& ch) { return launch_mrhs_choice<N, T>(a, ch, s); },
                     s, &c);
  if (rc != COARSE_OK) return rc;
  return launch_mrhs_choice<N, T>(a, c, s);
}

template <int N>
int launch_mrhs_n(const MrhsArgs& a, cudaStream_t s) {
  switch ((a.R + kMrhsTile - 1) / kMrhsTile) {
    case 1: return launch_mrhs_t<N, 1>(a, s);
    case 2: return launch_mrhs_t<N, 2>(a, s);
    case 3: return launch_mrhs_t<N, 3>(a, s);
    case 4:
      if constexpr (N == 32 || N == 48)
        if (a.tcblk) return launch_mrhs_t<N, 4>(a, s);
      break;
  }
  set_error("multi-RHS apply: %d columns in one pass", a.R);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace

int launch_pack_mrhs(const coarse_op* op, cudaStream_t s) {
  if (!op->mrhs.ptr) return COARSE_OK;
  if (op->umma.ptr) {
    const int rc = launch_pack_tc(op->blk[COARSE_PREC_BF16].ptr, op->umma.ptr, (long long)op->V * 5, op->n, s);
    if (rc != COARSE_OK) return rc;
  }
  const size_t total = (size_t)op->V * 5 * op->n * op->n;
  size_t grid = (total + 255) / 256;
  if (grid > (size_t)sm_count() * 16) grid = (size_t)sm_count() * 16;
  k_pack_mrhs<<<(int)grid, 256, 0, s>>>((const uint32_t*)op->blk[COARSE_PREC_BF16].ptr, (uint32_t*)op->mrhs.ptr,
                                        op->V, op->n);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_apply_mrhs_bf16(const coarse_op* op, const void* x, void* y, int nrhs, int adjoint, cudaStream_t s) {
  if (!op->mrhs.ptr) {
    set_error("multi-RHS apply needs BF16 blocks and max_nrhs > 1");
    return COARSE_ERR_INVALID_ARG;
  }
  if (((uintptr_t)x | (uintptr_t)y) & 15) {
    set_error("multi-RHS apply: x and y must be 16-byte aligned");
    return COARSE_ERR_INVALID_ARG;
  }
  const long long col = (long long)op->V * op->n;
  // passes of 16 columns where the tcgen05 kernel exists (its accumulators hold 16), else 12
  const int pass = op->umma.ptr ? kTcPass : kMrhsPass;
  for (int c0 = 0; c0 < nrhs; c0 += pass) {
    MrhsArgs a{};
    a.frag = (const uint4*)op->mrhs.ptr;
    a.nb = op->nb;
    a.x = (const float2*)x + c0 * col;
    a.xb = (const uint2*)op->mrhs_x.ptr;
    a.y = (float2*)y + c0 * col;
    a.ldx = a.ldy = col;
    a.R = nrhs - c0 < pass ? nrhs - c0 : pass;
    a.tcblk = op->umma.ptr;
    a.V = op->V;
    a.mu = (float)(adjoint ? -op->mu : op->mu);
    a.adj = adjoint;
    a.err = op->apply_cnt + op->V;
    int rc;
    switch (op->n) {
      case 16: rc = launch_mrhs_n<16>(a, s); break;
      case 32: rc = launch_mrhs_n<32>(a, s); break;
      case 48: rc = launch_mrhs_n<48>(a, s); break;
      default: set_error("multi-RHS apply: unsupported n = %d", op->n); return COARSE_ERR_INVALID_ARG;
    }
    if (rc != COARSE_OK) return rc;
  }
  return COARSE_OK;
}

}  // namespace coarse
