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
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "apply_core.cuh"
#include "batch.cuh"
#include "pipe.cuh"
#include "tune.cuh"

namespace coarse {

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

namespace {

template <int N, class BT, class VT, class AC>
__global__ void __launch_bounds__(128) k_apply(ApplyArgs a) {
  if (a.stop != nullptr && *a.stop) return;
  __shared__ AC ys[4][N];
  const int warp = threadIdx.x >> 5;
  const int site = blockIdx.x * 4 + warp;
  if (site >= a.V) return;  // warp-uniform
  apply_site<N, BT, VT, AC>(a, site, ys[warp]);
}

// ------------------------------------------------------------------------------------------
// TMA-staged variant for FP32 / BF16 blocks.  Same push-pull arithmetic as k_apply, but every
// stored block (one contiguous n*n chunk) is brought into shared memory by a 1D bulk copy
// (cp.async.bulk, completion on an mbarrier), S blocks ahead of the block being computed, so a
// warp keeps several blocks in flight without holding them in registers.  Persistent grid: warp
// w of W_total handles the contiguous site range [V*w/W_total, V*(w+1)/W_total).
// Every mbarrier wait is bounded: on expiry the kernel raises *a.err, drains its own copies (also
// bounded) and returns.
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
    // Packed FP32x2 accumulation: with e = (re, im) of a block entry used as-is,
    //   forward   yf += e*w      : F1 += e (.) (w.x, w.x),  F2 += e (.) (w.y, w.y)
    //             -> yf = (F1.x - F2.y, F2.x + F1.y)
    //   transpose yb += conj(e)*x : B1 += e (.) (x.x, x.x),  B2 += e (.) (x.y, x.y)
    //             -> yb = (B1.x + B2.y, B2.x - B1.y)
    // so each entry costs four __ffma2_rn and no operand shuffling.
    float2 xr1[KR], xr2[KR];
    float2 F1[KR], F2[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) { F1[k] = make_float2(0.f, 0.f); F2[k] = make_float2(0.f, 0.f); }
    const AT so = adj ? AT(1) : st;
#pragma unroll 1
    for (int b = 0; b < 5; ++b, ++it) {
      const int sidx = it % S;
      if (!mbar_wait(bar + sidx, (uint32_t)((it / S) & 1))) ok = false;
      if (!__all_sync(0xffffffffu, ok)) break;
      const VT* vs = reinterpret_cast<const VT*>(stage0 + (size_t)sidx * SB + BB);
      float2 w1[CPL], w2[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const VT v = vs[t * CPL + c];
        const AT sc = adj ? st : AT(1);
        w1[c] = make_float2(sc * v.x, sc * v.x);
        w2[c] = make_float2(sc * v.y, sc * v.y);
      }
      if (b == 0) {
        // own vector: its rows feed the pushes of the four hop blocks
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const VT v = vs[4 * k + g];
          const AT sk = (adj || 4 * k + g < NV) ? AT(1) : AT(-1);
          xr1[k] = make_float2(sk * v.x, sk * v.x);
          xr2[k] = make_float2(sk * v.y, sk * v.y);
        }
      }
      const BT* blk = reinterpret_cast<const BT*>(stage0 + (size_t)sidx * SB) + g * N + t * CPL;
      float2 B1[CPL], B2[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) { B1[c] = make_float2(0.f, 0.f); B2[c] = make_float2(0.f, 0.f); }
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        AC e[CPL];
        SmemRow<BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          F1[k] = __ffma2_rn(e[c], w1[c], F1[k]);
          F2[k] = __ffma2_rn(e[c], w2[c], F2[k]);
          if (b > 0) {
            B1[c] = __ffma2_rn(e[c], xr1[k], B1[c]);
            B2[c] = __ffma2_rn(e[c], xr2[k], B2[c]);
          }
        }
      }
      AC yb[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) yb[c] = make_float2(B1[c].x + B2[c].y, B2[c].x - B1[c].y);
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
    AC yf[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      yf[k] = make_float2(F1[k].x - F2[k].y, F2[k].x + F1[k].y);
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

// ------------------------------------------------------------------------------------------
// Batched stencil: one launch applies D_c for every solve of an n-group.  Warp g of the flat
// grid takes global site g, finds its solve through the site prefix sums and runs the same
// per-site push-pull body as k_apply with that solve's operator, vectors and scratch.
template <int N, class BT>
__global__ void __launch_bounds__(128) kb_apply(BApply b) {
  __shared__ float2 ys[4][N];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * 4 + warp;
  if (g >= b.total) return;
  const int k = find_solve(b.site_off, b.count, g);
  const BSolve& s = b.S[b.sidx[k]];
  if (!bgate(s, b.gate)) return;  // uniform for all sites of the solve
  const int step = *b.step;
  ApplyArgs a;
  a.blocks = b.poly_blocks ? s.blk_poly : s.blk;
  a.nb = s.nb;
  a.V = s.V;
  a.mu = s.mu;
  a.x = bsel(s, b.xsel, step);
  a.y = bsel(s, b.ysel, step);
  a.z = nullptr;
  a.acc = s.acc;
  a.coef = s.polyc + b.coef_off;
  a.mode = b.mode;
  a.adjoint = 0;
  a.stop = nullptr;
  a.part = s.part;
  a.push = s.push;
  a.cnt = s.cnt;
  a.err = s.cnt + s.V;
  apply_site<N, BT, float2, float2>(a, g - b.site_off[k], ys[warp]);
}

// FP64 residual of every not-yet-converged solve: r64 = b64 - D x64.
template <int N>
__global__ void __launch_bounds__(128) kb_residual64(BApply b, const double2* coef) {
  __shared__ double2 ys[4][N];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * 4 + warp;
  if (g >= b.total) return;
  const int k = find_solve(b.site_off, b.count, g);
  const BSolve& s = b.S[b.sidx[k]];
  if (!bgate(s, b.gate)) return;
  ApplyArgs a;
  a.blocks = s.blk64;
  a.nb = s.nb;
  a.V = s.V;
  a.mu = s.mu;
  a.x = s.x64;
  a.y = s.r64;
  a.z = s.b64;
  a.acc = nullptr;
  a.coef = coef;
  a.mode = APPLY_AXPBY;
  a.adjoint = 0;
  a.stop = nullptr;
  a.part = s.part64;
  a.push = (char*)s.part64 + (size_t)s.Nf * sizeof(double2);
  a.cnt = s.cnt;
  a.err = s.cnt + s.V;
  apply_site<N, double2, double2, double2>(a, g - b.site_off[k], ys[warp]);
}

}  // namespace

// FP32 / BF16: the autotuner picks, per (precision, n, lattice-size bucket), between the
// TMA-staged persistent kernel (candidate 0, the default) and the register push-pull kernel
// (candidate 1).  Candidates are timed in plain mode into a scratch output, so that an epilogue
// that accumulates (the polynomial chain) never runs twice; decisions are cached per process.
template <class BT>
int launch_tuned(int prec, int n, const ApplyArgs& a, cudaStream_t s) {
  const int ni = n / 16 - 1, vb = std::min(tune_bucket(a.V), 31);
  if (ni < 0 || ni > 2) {
    set_error("coarse_apply: unsupported n = %d (nv must be 8, 16 or 24)", n);
    return COARSE_ERR_INVALID_ARG;
  }
  int choice = tune_fast_get(0, prec, ni, vb);
  if (choice < 0) {
    char key[64];
    snprintf(key, sizeof(key), "apply/p%d/n%d/v%d", prec, n, vb);
    void* scratch = nullptr;
    auto run = [&](const TuneChoice& c) -> int {
      if (!scratch && cudaMalloc(&scratch, sizeof(float2) * (size_t)a.V * n) != cudaSuccess) {
        cudaGetLastError();
        set_error("coarse_apply: autotuner scratch allocation failed");
        return COARSE_ERR_OOM;
      }
      ApplyArgs t = a;
      t.mode = APPLY_PLAIN;
      t.y = scratch;
      t.z = nullptr;
      t.acc = nullptr;
      t.coef = nullptr;
      t.stop = nullptr;
      return c.a == 1 ? launch_t<BT, float2, float2>(n, t, s) : launch_tma<BT>(n, t, s);
    };
    TuneChoice c;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const int rc = tune_pick(key, {TuneChoice{0, 0, 0}, TuneChoice{1, 0, 0}}, run, s, &c);
    if (scratch) {
      cudaStreamSynchronize(s);
      cudaFree(scratch);
    }
    if (rc != COARSE_OK) return rc;
    if (cap == cudaStreamCaptureStatusNone) tune_fast_put(0, prec, ni, vb, c.a);
    choice = c.a;
  }
  return choice == 1 ? launch_t<BT, float2, float2>(n, a, s) : launch_tma<BT>(n, a, s);
}

int launch_apply(int prec, int n, const ApplyArgs& a, cudaStream_t s) {
  if (a.V <= 0) return COARSE_OK;
  switch (prec) {
    case COARSE_PREC_FP64: return launch_t<double2, double2, double2>(n, a, s);
    case COARSE_PREC_FP32: return launch_tuned<float2>(prec, n, a, s);
    case COARSE_PREC_BF16: return launch_tuned<cbf16>(prec, n, a, s);
  }
  set_error("coarse_apply: unknown precision %d", prec);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace coarse

namespace coarse {

int launch_bapply(int prec, int n, const BApply& b, cudaStream_t s) {
  if (b.total <= 0) return COARSE_OK;
  const int grid = (b.total + 3) / 4;
  if (prec == COARSE_PREC_FP32) {
    switch (n) {
      case 16: kb_apply<16, float2><<<grid, 128, 0, s>>>(b); break;
      case 32: kb_apply<32, float2><<<grid, 128, 0, s>>>(b); break;
      case 48: kb_apply<48, float2><<<grid, 128, 0, s>>>(b); break;
      default: set_error("batched apply: unsupported n = %d", n); return COARSE_ERR_INVALID_ARG;
    }
  } else {
    switch (n) {
      case 16: kb_apply<16, cbf16><<<grid, 128, 0, s>>>(b); break;
      case 32: kb_apply<32, cbf16><<<grid, 128, 0, s>>>(b); break;
      case 48: kb_apply<48, cbf16><<<grid, 128, 0, s>>>(b); break;
      default: set_error("batched apply: unsupported n = %d", n); return COARSE_ERR_INVALID_ARG;
    }
  }
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_bapply64_residual(int n, const BApply& b, cudaStream_t s) {
  if (b.total <= 0) return COARSE_OK;
  const int grid = (b.total + 3) / 4;
  // {-1, +1} for r = -D x + b lives right after the step counter (see the batch layout)
  const double2* coef = reinterpret_cast<const double2*>(b.step + 4);
  switch (n) {
    case 16: kb_residual64<16><<<grid, 128, 0, s>>>(b, coef); break;
    case 32: kb_residual64<32><<<grid, 128, 0, s>>>(b, coef); break;
    case 48: kb_residual64<48><<<grid, 128, 0, s>>>(b, coef); break;
    default: set_error("batched residual: unsupported n = %d", n); return COARSE_ERR_INVALID_ARG;
  }
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace coarse
