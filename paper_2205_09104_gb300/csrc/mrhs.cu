// Multi-right-hand-side apply Y = D_c X on tensor cores (BF16 blocks and vector fragments,
// FP32 accumulation), and the repacking of the BF16 blocks into the fragment-native layout
// it reads.  The per-block tensor-core computation is in mrhs_core.cuh.
//
// Staging.  A CTA owns P consecutive sites at a time (P = 4, 2, 1 for n = 16, 32, 48) and walks
// the 9 blocks of Eq. (6) for them: item b = 0 self, 1..4 forward hop mu = b-1 (block of x, vector
// of x+mu), 5..8 backward hop mu = b-5 (block of x-mu, vector of x-mu).  A pre-pass
// (k_pack_mrhs_x) rounds the R complex64 columns to BF16 B fragments, contiguous per site, so
// that one producer warp brings each item's P blocks and P vector sets into a ring of S
// shared-memory stages with 2P 1D bulk copies completing on the stage's "full" mbarrier;
// P * n/16 consumer warps (site p, row tile rt) run the tensor-core products from shared memory
// and release the stage on its "empty" mbarrier.  Every byte is loaded once per CTA.  All waits
// are bounded (pipe.cuh): on expiry the kernel raises *err, the producer drains its copies in
// flight, and all warps return.
#include <cstdio>
#include <vector>

#include "mrhs_core.cuh"
#include "pipe.cuh"
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

// complex64 columns x + q*ldx (q < R) -> fragment-native BF16 B operands (layout in mrhs_core.cuh),
// zeros for the columns R .. 4T-1 of the last tile.
__global__ void k_pack_mrhs_x(const float2* __restrict__ x, long long ldx, int R, int T, int V, int n,
                              uint32_t* __restrict__ xb) {
  const int NT = n / 16;
  const size_t total = (size_t)V * T * NT * 64;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int w = (int)(i & 1), lane = (int)((i >> 1) & 31);
    size_t rest = i >> 6;
    const int kt = (int)(rest % NT);
    rest /= NT;
    const int tl = (int)(rest % T);
    const size_t site = rest / T;
    const int g = lane >> 2, t = lane & 3;
    const int q = kMrhsTile * tl + (g >> 1);
    uint32_t v = 0u;
    if (q < R) {
      const float4 e = __ldg(reinterpret_cast<const float4*>(x + q * ldx + site * n + 16 * kt + 2 * t + 8 * w));
      v = (g & 1) ? bf2_bits(e.y, e.w) : bf2_bits(e.x, e.z);
    }
    xb[i] = v;
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
};

template <int N, int P> struct MrhsShape {
  static constexpr int NT = N / 16;
  static constexpr int WC = P * NT;            // consumer warps
  static constexpr int THREADS = (WC + 1) * 32;
  static constexpr uint32_t BLK = 4u * N * N;  // bytes of one block
};

// P sites per stage (template), S stages (runtime); see the file comment.
template <int N, int T, int P>
__global__ void __launch_bounds__(MrhsShape<N, P>::THREADS) k_apply_mrhs(MrhsArgs a) {
  using Sh = MrhsShape<N, P>;
  constexpr int NT = Sh::NT, WC = Sh::WC;
  constexpr uint32_t BLK = Sh::BLK, VB = T * NT * 256u;  // bytes of one block / one site's vector fragments
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = a.S;
  const uint32_t SB = a.SB;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
  uint64_t* empty = full + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = (a.V + P - 1) / P;
  const int my_groups = (int)blockIdx.x < ngroups ? (ngroups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int items = my_groups * 9;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, WC);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == WC) {  // ---------------------------------------------------------- producer
    // lane p < P issues the block copy of site p of the group, lane P + p its vector copy; both
    // keep the site's neighbour row (prefetched one group ahead) in registers.
    const int p = lane < P ? lane : lane - P;
    const bool active = lane < 2 * P;
    int4 nb_lo = make_int4(0, 0, 0, 0), nb_hi = nb_lo, nx_lo = nb_lo, nx_hi = nb_lo;
    auto fetch = [&](int grp, int4& lo, int4& hi) {
      const int x = grp * P + p;
      if (active && grp < ngroups && x < a.V) {
        lo = __ldg(reinterpret_cast<const int4*>(a.nb + x * 8));
        hi = __ldg(reinterpret_cast<const int4*>(a.nb + x * 8 + 4));
      }
    };
    fetch((int)blockIdx.x, nx_lo, nx_hi);
    int ok = 1;
    int it = 0;
    for (; it < items; ++it) {
      const int slot = it % S;
      const int grp = (int)blockIdx.x + (it / 9) * (int)gridDim.x, b = it % 9;
      if (b == 0) {
        nb_lo = nx_lo;
        nb_hi = nx_hi;
        fetch(grp + (int)gridDim.x, nx_lo, nx_hi);
      }
      if (it >= S && lane == 0) ok = mbar_wait_suspend(empty + slot, (uint32_t)((it / S - 1) & 1)) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      const int x0 = grp * P;
      const int np = a.V - x0 < P ? a.V - x0 : P;
      unsigned char* st = smem + (size_t)slot * SB;
      if (lane == 0) mbar_expect_tx(full + slot, (uint32_t)np * (BLK + VB));
      __syncwarp();
      if (active && p < np) {
        const int x = x0 + p;
        // source site of the vector: x (self), x + mu (forward hop), x - mu (backward hop)
        int src = x;
        switch (b) {
          case 1: src = nb_lo.x; break;
          case 2: src = nb_lo.y; break;
          case 3: src = nb_lo.z; break;
          case 4: src = nb_lo.w; break;
          case 5: src = nb_hi.x; break;
          case 6: src = nb_hi.y; break;
          case 7: src = nb_hi.z; break;
          case 8: src = nb_hi.w; break;
        }
        if (lane < P) {
          const size_t blkid = b < 5 ? (size_t)x * 5 + b : (size_t)src * 5 + 1 + (b - 5);
          bulk_g2s(st + p * BLK, a.frag + blkid * (BLK / 16), BLK, full + slot);
        } else {
          bulk_g2s(st + P * BLK + p * VB, a.xb + (size_t)src * (VB / 8), VB, full + slot);
        }
      }
    }
    if (!ok && lane == 0) {
      atomicExch(a.err, 1);
      // drain the bulk copies this CTA still has in flight (bounded) before it exits
      for (int j = it - S < 0 ? 0 : it - S; j < it; ++j) mbar_wait(full + (j % S), (uint32_t)((j / S) & 1));
    }
    return;
  }

  // ---------------------------------------------------------------------------------- consumers
  const int p = warp / NT, rt = warp % NT;
  const int t = lane & 3, g = lane >> 2;
  MrhsAcc<T> acc;
  acc.zero();
  int ok = 1;
  for (int it = 0; it < items; ++it) {
    const int slot = it % S;
    if (!mbar_wait_suspend(full + slot, (uint32_t)((it / S) & 1))) ok = 0;
    if (!__all_sync(0xffffffffu, ok)) break;
    const int grp = (int)blockIdx.x + (it / 9) * (int)gridDim.x, b = it % 9;
    const int x = grp * P + p;
    const bool valid = x < a.V;
    const unsigned char* st = smem + (size_t)slot * SB;
    if (valid)
      mrhs_block<N, T>(reinterpret_cast<const uint4*>(st + p * BLK),
                       reinterpret_cast<const uint2*>(st + P * BLK + p * VB), rt, b >= 5, a.adj, acc);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + slot);
    if (b == 8) {
      if (valid) {
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
      acc.zero();
    }
  }
  if (!ok && lane == 0) atomicExch(a.err, 1);
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
  a.SB = (uint32_t)P * (Sh::BLK + (uint32_t)T * Sh::NT * 256u);
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
template <int N>
std::vector<TuneChoice> mrhs_candidates() {
  std::vector<TuneChoice> c;
  const int def_p = N == 16 ? 4 : (N == 32 ? 2 : 1);
  const int ps[3] = {N == 16 ? 2 : 1, N == 16 ? 4 : 2, N == 16 ? 8 : 4};
  c.push_back({def_p, 0, 0});
  for (int P : ps) {
    if (P * (N / 16) > 8) continue;
    for (int S : {3, 5, 8})
      if (!(P == def_p && S == 0)) c.push_back({P, S, 0});
  }
  return c;
}

template <int N, int T>
int launch_mrhs_choice(const MrhsArgs& a, const TuneChoice& c, cudaStream_t s) {
  switch (c.a) {
    case 1: return launch_mrhs_cfg<N, T, 1>(a, c.b, s);
    case 2: return launch_mrhs_cfg<N, T, 2>(a, c.b, s);
    case 4: return launch_mrhs_cfg<N, T, 4>(a, c.b, s);
    case 8:
      if constexpr (N == 16) return launch_mrhs_cfg<N, T, 8>(a, c.b, s);
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
  int rc = tune_pick(key, mrhs_candidates<N>(), [&](const TuneChoice& ch) { return launch_mrhs_choice<N, T>(a, ch, s); },
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
  }
  set_error("multi-RHS apply: %d columns in one pass", a.R);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace

int launch_pack_mrhs(const coarse_op* op, cudaStream_t s) {
  if (!op->mrhs.ptr) return COARSE_OK;
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
  for (int c0 = 0; c0 < nrhs; c0 += kMrhsPass) {
    MrhsArgs a{};
    a.frag = (const uint4*)op->mrhs.ptr;
    a.nb = op->nb;
    a.x = (const float2*)x + c0 * col;
    a.xb = (const uint2*)op->mrhs_x.ptr;
    a.y = (float2*)y + c0 * col;
    a.ldx = a.ldy = col;
    a.R = nrhs - c0 < kMrhsPass ? nrhs - c0 : kMrhsPass;
    {
      const int T = (a.R + kMrhsTile - 1) / kMrhsTile;
      const size_t total = (size_t)op->V * T * (op->n / 16) * 64;
      size_t grid = (total + 255) / 256;
      if (grid > (size_t)sm_count() * 16) grid = (size_t)sm_count() * 16;
      k_pack_mrhs_x<<<(int)grid, 256, 0, s>>>(a.x, a.ldx, a.R, T, op->V, op->n, (uint32_t*)op->mrhs_x.ptr);
      note_launch();
      COARSE_CUDA(cudaGetLastError());
    }
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
