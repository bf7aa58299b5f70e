// Coarse stencil apply y = D_c x (Sec. 2.2), gamma5-compressed storage.
//
// Storage: blocks[V][5][n][n] row-major complex, block 0 = self A_x, blocks
// 1..4 = forward hops F_{x,mu} = D_c[x, x+mu].  The backward hop of site x in
// direction mu is D_c[x, x-mu] = sigma3 F_{x-mu,mu}^H sigma3 (Sec. 4.2 on the
// coarse level), so each stored hop block serves two sites.  The kernel reads
// every stored block exactly once (push-pull, see k_apply below).
//
// Thread mapping: one warp per site.  Lane l = 8*g + t, g = row group (0..3),
// t = column chunk (0..7).  For block row i = 4k + g the lane reads the CPL =
// n/8 consecutive entries in columns t*CPL .. t*CPL+CPL-1, so a warp reads 4
// whole rows per step in one coalesced sweep of the row-major block.  The
// lane's columns are the same for every row, hence from the same registers
//   forward use  y_i  += F_ij w_j : n/4 row partial sums per lane, reduced over t
//   transposed   y'_j += conj(F_ij) w'_i : CPL column sums per lane, reduced over g
// without shared-memory staging of the block.
#include "common.cuh"

namespace coarse {
namespace {

// BF16 complex (re, im) in 32 bits -> float2
__device__ __forceinline__ float2 bf2f(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

template <class VT, class AC, int CPL>
__device__ __forceinline__ void load_vec(const VT* p, AC (&w)[CPL]) {
#pragma unroll
  for (int c = 0; c < CPL; ++c) { VT v = p[c]; w[c].x = v.x; w[c].y = v.y; }
}
template <class VT, class AC, int CPL>
__device__ __forceinline__ void store_vec(VT* p, const AC (&w)[CPL]) {
#pragma unroll
  for (int c = 0; c < CPL; ++c) { VT v; v.x = w[c].x; v.y = w[c].y; p[c] = v; }
}

// Streaming (read-once) block loads: evict-first so that the per-site pushes stay in L2.
template <class T> __device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

template <class AC, class BT> struct LoadS;
template <> struct LoadS<double2, double2> {
  template <int CPL> __device__ __forceinline__ static void row(const double2* p, double2 (&e)[CPL]) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) e[c] = ld_stream(p + c);
  }
};
template <> struct LoadS<float2, float2> {
  template <int CPL> __device__ __forceinline__ static void row(const float2* p, float2 (&e)[CPL]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      float4 v = ld_stream(q + c);
      e[2 * c] = make_float2(v.x, v.y);
      e[2 * c + 1] = make_float2(v.z, v.w);
    }
  }
};
template <> struct LoadS<float2, cbf16> {
  template <int CPL> __device__ __forceinline__ static void row(const cbf16* p, float2 (&e)[CPL]) {
    if constexpr ((CPL * 4) % 16 == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 4; ++c) {
        uint4 v = ld_stream(q + c);
        e[4 * c] = bf2f(v.x); e[4 * c + 1] = bf2f(v.y); e[4 * c + 2] = bf2f(v.z); e[4 * c + 3] = bf2f(v.w);
      }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 2; ++c) {
        uint2 v = ld_stream(q + c);
        e[2 * c] = bf2f(v.x); e[2 * c + 1] = bf2f(v.y);
      }
    }
  }
};

template <class AC> __device__ __forceinline__ AC ld_cg(const AC* p);
template <> __device__ __forceinline__ float2 ld_cg<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ld_cg<double2>(const double2* p) { return __ldcg(p); }

// Finish the sites flagged in `fin` (bit 0: `site`, bit 1+mu: its forward neighbour mu):
//   y_z = P_z + T_0[z-0] + T_1[z-1] + T_2[z-2] + T_3[z-3] + i mu sigma3 v_z, then the epilogue.
// Called by the 8 lanes of row group 0 (lane t owns columns t*CPL ...).
template <int N, class VT, class AC>
__device__ __forceinline__ void finish_sites(const ApplyArgs& a, int site, int fin, int t,
                                             decltype(AC{}.x) st, const AC* Pb, const AC* Tb) {
  constexpr int CPL = N / 8;
  using AT = decltype(AC{}.x);
  const int V = a.V;
  const double2 c0d = a.mode != APPLY_PLAIN ? a.coef[0] : make_double2(0.0, 0.0);
  const double2 c1d = a.mode != APPLY_PLAIN ? a.coef[1] : make_double2(0.0, 0.0);
  const double2 c2d = a.mode == APPLY_POLY_FIRST ? a.coef[2] : make_double2(0.0, 0.0);
  const AC c0{AT(c0d.x), AT(c0d.y)}, c1{AT(c1d.x), AT(c1d.y)}, c2{AT(c2d.x), AT(c2d.y)};
  const VT* X = static_cast<const VT*>(a.x);
#pragma unroll 1
  for (int q = 0; q < 5; ++q) {
    if (!(fin & (1 << q))) continue;
    const int z = q == 0 ? site : __ldg(a.nb + site * 8 + (q - 1));
    AC r[CPL], xs[CPL];
    load_vec<VT, AC, CPL>(X + (size_t)z * N + t * CPL, xs);
#pragma unroll
    for (int c = 0; c < CPL; ++c) r[c] = ld_cg(Pb + (size_t)z * N + t * CPL + c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int from = __ldg(a.nb + z * 8 + 4 + mu);
      const AC* srcp = Tb + ((size_t)mu * V + from) * N + t * CPL;
#pragma unroll
      for (int c = 0; c < CPL; ++c) r[c] = cadd(r[c], ld_cg(srcp + c));
    }
    const AT m = AT(a.mu) * st;  // + i mu sigma3 v
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      r[c].x -= m * xs[c].y;
      r[c].y += m * xs[c].x;
    }
    VT* Y = static_cast<VT*>(a.y) + (size_t)z * N + t * CPL;
    if (a.mode == APPLY_PLAIN) {
      store_vec<VT, AC, CPL>(Y, r);
    } else if (a.mode == APPLY_AXPBY) {
      AC zz[CPL];
      load_vec<VT, AC, CPL>(static_cast<const VT*>(a.z) + (size_t)z * N + t * CPL, zz);
#pragma unroll
      for (int c = 0; c < CPL; ++c) r[c] = cadd(cmul(c0, r[c]), cmul(c1, zz[c]));
      store_vec<VT, AC, CPL>(Y, r);
    } else {
      // polynomial chain: s' = s - c0 * D s ; acc = acc + c1 * s'  (first step: acc = c2 * s + c1 * s')
      VT* Acc = static_cast<VT*>(a.acc) + (size_t)z * N + t * CPL;
      AC ac[CPL];
      if (a.mode == APPLY_POLY_FIRST) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) ac[c] = cmul(c2, xs[c]);
      } else {
        load_vec<VT, AC, CPL>(Acc, ac);
      }
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        r[c] = csub(xs[c], cmul(c0, r[c]));
        ac[c] = cadd(ac[c], cmul(c1, r[c]));
      }
      store_vec<VT, AC, CPL>(Y, r);
      store_vec<VT, AC, CPL>(Acc, ac);
    }
    if (t == 0) a.cnt[z] = 0;
  }
}

// Push-pull apply.  The warp of site x reads its 5 stored blocks once:
//   pull  P_x      = A_x v_x + sum_mu F_{x,mu} v_{x+mu}            (row sums)
//   push  T_mu[x]  = sigma3 F_{x,mu}^H sigma3 v_x                  (column sums, for site x+mu)
// and writes them to scratch.  Each site receives 5 contributions (its own
// pull and one push per direction from x-mu); a per-site counter tells the
// warp that delivers the 5th contribution to finish the site:
//   y_z = P_z + T_0[z-0] + T_1[z-1] + T_2[z-2] + T_3[z-3] + i mu sigma3 v_z, then the epilogue.
// The sum order is fixed, so results do not depend on which warp finishes.
// The finisher resets the counter to 0 for the next launch.  No thread ever
// waits for another.
template <int N, class BT, class VT, class AC>
__global__ void __launch_bounds__(128) k_apply(ApplyArgs a) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2;
  using AT = decltype(AC{}.x);
  if (a.stop != nullptr && *a.stop) return;
  __shared__ AC ys[4][N];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int site = blockIdx.x * 4 + warp;
  if (site >= a.V) return;  // warp-uniform
  const int g = lane >> 3, t = lane & 7;
  const int V = a.V;
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* X = static_cast<const VT*>(a.x);
  AC* Pb = static_cast<AC*>(a.part);
  AC* Tb = static_cast<AC*>(a.push);
  constexpr size_t BSZ = (size_t)N * N;
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);  // sigma3 of this lane's columns
  const int adj = a.adjoint;

  // own vector: the lane's columns (pull of the self block) and its rows (pushes)
  AC w0[CPL], xr[KR];
  load_vec<VT, AC, CPL>(X + (size_t)site * N + t * CPL, w0);
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const VT v = X[(size_t)site * N + 4 * k + g];
    const AT sk = (adj || 4 * k + g < NV) ? AT(1) : AT(-1);  // sigma3 on the push input
    xr[k].x = sk * AT(v.x);
    xr[k].y = sk * AT(v.y);
  }
  AC yf[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) yf[k] = AC{0, 0};
  {
    AC w[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) w[c] = adj ? cscale(w0[c], st) : w0[c];
    const BT* blk = B + (size_t)site * 5 * BSZ + g * N + t * CPL;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      AC e[CPL];
      LoadS<AC, BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) cfma(yf[k], e[c], w[c]);
    }
  }
  const AT so = adj ? AT(1) : st;  // sigma3 on the push output (columns)
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int src = __ldg(a.nb + site * 8 + mu);
    AC w[CPL];
    load_vec<VT, AC, CPL>(X + (size_t)src * N + t * CPL, w);
    if (adj) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) w[c] = cscale(w[c], st);
    }
    AC yb[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};
    const BT* blk = B + ((size_t)site * 5 + 1 + mu) * BSZ + g * N + t * CPL;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      AC e[CPL];
      LoadS<AC, BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        cfma(yf[k], e[c], w[c]);
        cfma_conj(yb[c], e[c], xr[k]);
      }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
#pragma unroll
      for (int off = 8; off < 32; off <<= 1) {
        yb[c].x += __shfl_xor_sync(0xffffffffu, yb[c].x, off);
        yb[c].y += __shfl_xor_sync(0xffffffffu, yb[c].y, off);
      }
    }
    if (g == 0) {
      AC* dst = Tb + ((size_t)mu * V + site) * N + t * CPL;
#pragma unroll
      for (int c = 0; c < CPL; ++c) dst[c] = cscale(yb[c], so);
    }
  }
#pragma unroll
  for (int k = 0; k < KR; ++k) {
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      yf[k].x += __shfl_xor_sync(0xffffffffu, yf[k].x, off);
      yf[k].y += __shfl_xor_sync(0xffffffffu, yf[k].y, off);
    }
  }
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const AT sr = (adj && 4 * k + g >= NV) ? AT(-1) : AT(1);
      ys[warp][4 * k + g] = cscale(yf[k], sr);
    }
  }
  __syncwarp();
  if (g == 0) {
    AC* dst = Pb + (size_t)site * N + t * CPL;
#pragma unroll
    for (int c = 0; c < CPL; ++c) dst[c] = ys[warp][t * CPL + c];
  }
  // publish: every lane fences its own stores, then lane 0 counts the 5 deliveries
  __threadfence();
  __syncwarp();
  int fin = 0;
  if (lane == 0) {
    if (atomicAdd(a.cnt + site, 1) == 4) fin |= 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
      if (atomicAdd(a.cnt + __ldg(a.nb + site * 8 + mu), 1) == 4) fin |= 2 << mu;
  }
  fin = __shfl_sync(0xffffffffu, fin, 0);
  if (fin == 0 || g != 0) return;
  __threadfence();
  finish_sites<N, VT, AC>(a, site, fin, t, st, Pb, Tb);
}

// ------------------------------------------------------------------------------------------
// TMA-staged variant for FP32 / BF16 blocks.  Same push-pull arithmetic as k_apply, but every
// stored block (one contiguous n*n chunk) is brought into shared memory by a 1D bulk copy
// (cp.async.bulk, completion on an mbarrier), S blocks ahead of the block being computed, so a
// warp keeps several blocks in flight without holding them in registers.  Persistent grid: warp
// w of W_total handles the contiguous site range [V*w/W_total, V*(w+1)/W_total).
// Every mbarrier wait is bounded: on expiry the kernel raises *a.err, drains its own copies (also
// bounded) and returns.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: true when the phase completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <class BT> struct SmemRow;
template <> struct SmemRow<float2> {
  template <int CPL> __device__ __forceinline__ static void row(const float2* p, float2 (&e)[CPL]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      const float4 v = q[c];
      e[2 * c] = make_float2(v.x, v.y);
      e[2 * c + 1] = make_float2(v.z, v.w);
    }
  }
};
template <> struct SmemRow<cbf16> {
  template <int CPL> __device__ __forceinline__ static void row(const cbf16* p, float2 (&e)[CPL]) {
    if constexpr ((CPL * 4) % 16 == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 4; ++c) {
        const uint4 v = q[c];
        e[4 * c] = bf2f(v.x); e[4 * c + 1] = bf2f(v.y); e[4 * c + 2] = bf2f(v.z); e[4 * c + 3] = bf2f(v.w);
      }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 2; ++c) {
        const uint2 v = q[c];
        e[2 * c] = bf2f(v.x); e[2 * c + 1] = bf2f(v.y);
      }
    }
  }
};

// Shared-memory pipeline shape: a stage holds one block plus the vector it multiplies
// (brought by the same mbarrier transaction).  Prefer 8 warps per CTA with >= 3 stages,
// then 6, 5, 4 warps; at most 6 stages; ~210 KB of stages.
template <int N, class BT> struct TmaCfg {
  static constexpr int kBlockBytes = N * N * (int)sizeof(BT);
  static constexpr int kVecBytes = N * 8;
  static constexpr int kStageBytes = kBlockBytes + kVecBytes;
  static constexpr int kBudget = 210 * 1024;
  static constexpr int stages_for(int w) { return kBudget / (w * kStageBytes); }
  static constexpr int kWarps = stages_for(8) >= 3 ? 8 : stages_for(6) >= 3 ? 6 : stages_for(5) >= 2 ? 5 : 4;
  static constexpr int kS0 = stages_for(kWarps);
  static constexpr int kStages = kS0 < 2 ? 2 : (kS0 > 6 ? 6 : kS0);
  static constexpr size_t kSmem =
      (size_t)kWarps * kStages * kStageBytes + kWarps * kStages * 8 + kWarps * N * 8 + 128;
};

template <int N, class BT>
__global__ void __launch_bounds__(32 * TmaCfg<N, BT>::kWarps, 1) k_apply_tma(ApplyArgs a) {
  using Cfg = TmaCfg<N, BT>;
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2, S = Cfg::kStages, W = Cfg::kWarps;
  constexpr uint32_t BB = Cfg::kBlockBytes, SB = Cfg::kStageBytes, VB = Cfg::kVecBytes;
  using AC = float2;
  using AT = float;
  using VT = float2;
  extern __shared__ __align__(128) unsigned char smem[];
  if (a.stop != nullptr && *a.stop) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, t = lane & 7;
  const long long gw = (long long)blockIdx.x * W + warp, nw = (long long)gridDim.x * W;
  const int V = a.V;
  const int s0 = (int)((long long)V * gw / nw), s1 = (int)((long long)V * (gw + 1) / nw);
  if (s0 >= s1) return;  // warp-uniform
  unsigned char* stage0 = smem + (size_t)warp * S * SB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)W * S * SB) + warp * S;
  AC* ys = reinterpret_cast<AC*>(smem + (size_t)W * S * SB + W * S * 8) + warp * N;
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* X = static_cast<const VT*>(a.x);
  AC* Pb = static_cast<AC*>(a.part);
  AC* Tb = static_cast<AC*>(a.push);
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);
  const int adj = a.adjoint;
  const int items = (s1 - s0) * 5;
  if (lane == 0) {
    for (int i = 0; i < S; ++i) mbar_init(bar + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // item it = (site s0 + it/5, block b = it%5): the block and the vector it multiplies
  // (own vector for the self block, neighbour x+mu for forward hop mu)
  auto issue = [&](int it) {
    if (it < items) {
      const int sidx = it % S;
      const int site_i = s0 + it / 5, b = it % 5;
      const size_t blkid = (size_t)site_i * 5 + b;
      const int vsite = b == 0 ? site_i : __ldg(a.nb + site_i * 8 + (b - 1));
      unsigned char* dst = stage0 + (size_t)sidx * SB;
      mbar_expect_tx(bar + sidx, SB);
      bulk_g2s(dst, B + blkid * (size_t)N * N, BB, bar + sidx);
      bulk_g2s(dst + BB, X + (size_t)vsite * N, VB, bar + sidx);
    }
  };
  if (lane == 0)
    for (int i = 0; i < S; ++i) issue(i);
  bool ok = true;
  int it = 0;
  for (int site = s0; site < s1; ++site) {
    AC xr[KR];
    AC yf[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) yf[k] = AC{0, 0};
    const AT so = adj ? AT(1) : st;
#pragma unroll 1
    for (int b = 0; b < 5; ++b, ++it) {
      const int sidx = it % S;
      if (!mbar_wait(bar + sidx, (uint32_t)((it / S) & 1))) ok = false;
      if (!__all_sync(0xffffffffu, ok)) break;
      const VT* vs = reinterpret_cast<const VT*>(stage0 + (size_t)sidx * SB + BB);
      AC w[CPL];
      load_vec<VT, AC, CPL>(vs + t * CPL, w);
      if (b == 0) {
        // own vector: its rows feed the pushes of the four hop blocks
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const VT v = vs[4 * k + g];
          const AT sk = (adj || 4 * k + g < NV) ? AT(1) : AT(-1);
          xr[k].x = sk * v.x;
          xr[k].y = sk * v.y;
        }
      }
      if (adj) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) w[c] = cscale(w[c], st);
      }
      const BT* blk = reinterpret_cast<const BT*>(stage0 + (size_t)sidx * SB) + g * N + t * CPL;
      AC yb[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        AC e[CPL];
        SmemRow<BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          cfma(yf[k], e[c], w[c]);
          if (b > 0) cfma_conj(yb[c], e[c], xr[k]);
        }
      }
      __syncwarp();  // every lane has finished reading this stage
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(it + S);
      }
      if (b > 0) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
#pragma unroll
          for (int off = 8; off < 32; off <<= 1) {
            yb[c].x += __shfl_xor_sync(0xffffffffu, yb[c].x, off);
            yb[c].y += __shfl_xor_sync(0xffffffffu, yb[c].y, off);
          }
        }
        if (g == 0) {
          AC* dst = Tb + ((size_t)(b - 1) * V + site) * N + t * CPL;
#pragma unroll
          for (int c = 0; c < CPL; ++c) dst[c] = cscale(yb[c], so);
        }
      }
    }
    if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
#pragma unroll
      for (int off = 1; off < 8; off <<= 1) {
        yf[k].x += __shfl_xor_sync(0xffffffffu, yf[k].x, off);
        yf[k].y += __shfl_xor_sync(0xffffffffu, yf[k].y, off);
      }
    }
    if (t == 0) {
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const AT sr = (adj && 4 * k + g >= NV) ? AT(-1) : AT(1);
        ys[4 * k + g] = cscale(yf[k], sr);
      }
    }
    __syncwarp();
    if (g == 0) {
      AC* dst = Pb + (size_t)site * N + t * CPL;
#pragma unroll
      for (int c = 0; c < CPL; ++c) dst[c] = ys[t * CPL + c];
    }
    __threadfence();
    __syncwarp();
    int fin = 0;
    if (lane == 0) {
      if (atomicAdd(a.cnt + site, 1) == 4) fin |= 1;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu)
        if (atomicAdd(a.cnt + __ldg(a.nb + site * 8 + mu), 1) == 4) fin |= 2 << mu;
    }
    fin = __shfl_sync(0xffffffffu, fin, 0);
    if (fin != 0 && g == 0) {
      __threadfence();
      finish_sites<N, VT, AC>(a, site, fin, t, st, Pb, Tb);
    }
    __syncwarp();
  }
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) {
      atomicExch(a.err, 1);
      // drain this warp's copies still in flight (bounded) before the CTA exits
      for (int j = it; j < items && j < it + S; ++j) mbar_wait(bar + (j % S), (uint32_t)((j / S) & 1));
    }
    __syncwarp();
  }
}

template <class BT, class VT, class AC>
int launch_t(int n, const ApplyArgs& a, cudaStream_t s) {
  const dim3 grid((a.V + 3) / 4), block(128);
  switch (n) {
    case 16: k_apply<16, BT, VT, AC><<<grid, block, 0, s>>>(a); break;
    case 32: k_apply<32, BT, VT, AC><<<grid, block, 0, s>>>(a); break;
    case 48: k_apply<48, BT, VT, AC><<<grid, block, 0, s>>>(a); break;
    default: set_error("coarse_apply: unsupported n = %d (nv must be 8, 16 or 24)", n); return COARSE_ERR_INVALID_ARG;
  }
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int N, class BT>
int launch_tma_n(const ApplyArgs& a, cudaStream_t s) {
  using Cfg = TmaCfg<N, BT>;
  static bool attr = false;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_apply_tma<N, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem));
    attr = true;
  }
  int ctas = sm_count();
  const int need = (a.V + Cfg::kWarps - 1) / Cfg::kWarps;
  if (need < ctas) ctas = need;
  k_apply_tma<N, BT><<<ctas, 32 * Cfg::kWarps, Cfg::kSmem, s>>>(a);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

template <class BT>
int launch_tma(int n, const ApplyArgs& a, cudaStream_t s) {
  switch (n) {
    case 16: return launch_tma_n<16, BT>(a, s);
    case 32: return launch_tma_n<32, BT>(a, s);
    case 48: return launch_tma_n<48, BT>(a, s);
  }
  set_error("coarse_apply: unsupported n = %d (nv must be 8, 16 or 24)", n);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace

int launch_apply(int prec, int n, const ApplyArgs& a, cudaStream_t s) {
  if (a.V <= 0) return COARSE_OK;
  switch (prec) {
    case COARSE_PREC_FP64: return launch_t<double2, double2, double2>(n, a, s);
    case COARSE_PREC_FP32: return launch_tma<float2>(n, a, s);
    case COARSE_PREC_BF16: return launch_tma<cbf16>(n, a, s);
  }
  set_error("coarse_apply: unknown precision %d", prec);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace coarse
