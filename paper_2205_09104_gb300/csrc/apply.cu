// Coarse stencil apply y = D_c x (Sec. 2.2), gamma5-compressed storage.
//
// Storage: blocks[V][5][n][n] row-major complex, block 0 = self A_x, blocks
// 1..4 = forward hops F_{x,mu} = D_c[x, x+mu].  The backward hop of site x in
// direction mu is D_c[x, x-mu] = sigma3 F_{x-mu,mu}^H sigma3 (Sec. 4.2 on the
// coarse level), so each stored hop block serves two sites.
//
// Thread mapping: one warp per site.  Lane l = 8*g + t, g = row group (0..3),
// t = column chunk (0..7).  For block row i = 4k + g the lane reads the CPL =
// n/8 consecutive entries in columns t*CPL .. t*CPL+CPL-1, so a warp reads 4
// whole rows per step in one coalesced sweep of the row-major block.  The
// lane's columns are the same for every row, hence
//   forward use  y_i  += F_ij w_j : n/4 row partial sums per lane, reduced over t
//   backward use y'_j += conj(F_ij) w'_i : CPL column sums per lane, reduced over g
// and one read of a block feeds either product without shared-memory staging.
#include "common.cuh"

namespace coarse {
namespace {

template <class AC, class BT> struct Load;

// FP64 blocks: one 16-byte load per complex
template <> struct Load<double2, double2> {
  template <int CPL> __device__ __forceinline__ static void row(const double2* p, double2 (&e)[CPL]) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) e[c] = __ldg(p + c);
  }
};
// FP32 blocks: 16-byte loads (CPL is even)
template <> struct Load<float2, float2> {
  template <int CPL> __device__ __forceinline__ static void row(const float2* p, float2 (&e)[CPL]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      float4 v = __ldg(q + c);
      e[2 * c] = make_float2(v.x, v.y);
      e[2 * c + 1] = make_float2(v.z, v.w);
    }
  }
};
// BF16 blocks: 16-byte loads when the lane chunk is 16-byte aligned, else 8-byte loads
__device__ __forceinline__ float2 bf2f(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <> struct Load<float2, cbf16> {
  template <int CPL> __device__ __forceinline__ static void row(const cbf16* p, float2 (&e)[CPL]) {
    if constexpr ((CPL * 4) % 16 == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 4; ++c) {
        uint4 v = __ldg(q + c);
        e[4 * c] = bf2f(v.x); e[4 * c + 1] = bf2f(v.y); e[4 * c + 2] = bf2f(v.z); e[4 * c + 3] = bf2f(v.w);
      }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
      for (int c = 0; c < CPL / 2; ++c) {
        uint2 v = __ldg(q + c);
        e[2 * c] = bf2f(v.x); e[2 * c + 1] = bf2f(v.y);
      }
    }
  }
};

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

template <int N, class BT, class VT, class AC>
__global__ void __launch_bounds__(128) k_apply(ApplyArgs a) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2;
  using AT = decltype(AC{}.x);
  if (a.stop != nullptr && *a.stop) return;
  __shared__ AC ys[4][N];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int site = blockIdx.x * 4 + warp;
  if (site >= a.V) return;
  const int g = lane >> 3, t = lane & 7;
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* X = static_cast<const VT*>(a.x);
  constexpr size_t BSZ = (size_t)N * N;
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);  // sigma3 of this lane's columns
  const int adj = a.adjoint;

  AC yf[KR], yb[CPL], xs[CPL];
#pragma unroll
  for (int k = 0; k < KR; ++k) yf[k] = AC{0, 0};
#pragma unroll
  for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};

  // self and forward hops: y_i += B_ij w_j
#pragma unroll 1
  for (int b = 0; b < 5; ++b) {
    const int src = (b == 0) ? site : __ldg(a.nb + site * 8 + (b - 1));
    AC w[CPL];
    load_vec<VT, AC, CPL>(X + (size_t)src * N + t * CPL, w);
    if (b == 0) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) xs[c] = w[c];
    }
    if (adj) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) w[c] = cscale(w[c], st);
    }
    const BT* blk = B + ((size_t)site * 5 + b) * BSZ + g * N + t * CPL;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      AC e[CPL];
      Load<AC, BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) cfma(yf[k], e[c], w[c]);
    }
  }
  // backward hops: y'_j += conj(F_ij) s_i x_i, F = forward hop mu of site x - mu
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int xm = __ldg(a.nb + site * 8 + 4 + mu);
    const BT* blk = B + ((size_t)xm * 5 + 1 + mu) * BSZ + g * N + t * CPL;
    const VT* xv = X + (size_t)xm * N + g;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      VT v = xv[4 * k];
      AC wr;
      const AT sk = (adj || 4 * k + g < NV) ? AT(1) : AT(-1);
      wr.x = sk * AT(v.x);
      wr.y = sk * AT(v.y);
      AC e[CPL];
      Load<AC, BT>::template row<CPL>(blk + (size_t)k * 4 * N, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) cfma_conj(yb[c], e[c], wr);
    }
  }
  // row sums over the 8 column chunks, column sums over the 4 row groups
#pragma unroll
  for (int k = 0; k < KR; ++k) {
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      yf[k].x += __shfl_xor_sync(0xffffffffu, yf[k].x, off);
      yf[k].y += __shfl_xor_sync(0xffffffffu, yf[k].y, off);
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
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const AT sr = (adj && 4 * k + g >= NV) ? AT(-1) : AT(1);
      ys[warp][4 * k + g] = cscale(yf[k], sr);
    }
  }
  __syncwarp();
  if (g != 0) return;
  const AT so = adj ? AT(1) : st;
  AC r[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    r[c] = cadd(ys[warp][t * CPL + c], cscale(yb[c], so));
    // + i mu sigma3 x
    const AT m = AT(a.mu) * st;
    r[c].x -= m * xs[c].y;
    r[c].y += m * xs[c].x;
  }
  VT* Y = static_cast<VT*>(a.y) + (size_t)site * N + t * CPL;
  if (a.mode == APPLY_PLAIN) {
    store_vec<VT, AC, CPL>(Y, r);
    return;
  }
  const double2 c0d = a.coef[0], c1d = a.coef[1];
  const AC c0{AT(c0d.x), AT(c0d.y)}, c1{AT(c1d.x), AT(c1d.y)};
  if (a.mode == APPLY_AXPBY) {
    AC zz[CPL];
    load_vec<VT, AC, CPL>(static_cast<const VT*>(a.z) + (size_t)site * N + t * CPL, zz);
#pragma unroll
    for (int c = 0; c < CPL; ++c) r[c] = cadd(cmul(c0, r[c]), cmul(c1, zz[c]));
    store_vec<VT, AC, CPL>(Y, r);
    return;
  }
  // polynomial chain: s' = s - c0 * D s ; acc = acc + c1 * s'  (first step: acc = c2 * s + c1 * s')
  VT* Acc = static_cast<VT*>(a.acc) + (size_t)site * N + t * CPL;
  AC ac[CPL];
  if (a.mode == APPLY_POLY_FIRST) {
    const double2 c2d = a.coef[2];
    const AC c2{AT(c2d.x), AT(c2d.y)};
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

}  // namespace

int launch_apply(int prec, int n, const ApplyArgs& a, cudaStream_t s) {
  if (a.V <= 0) return COARSE_OK;
  switch (prec) {
    case COARSE_PREC_FP64: return launch_t<double2, double2, double2>(n, a, s);
    case COARSE_PREC_FP32: return launch_t<float2, float2, float2>(n, a, s);
    case COARSE_PREC_BF16: return launch_t<cbf16, float2, float2>(n, a, s);
  }
  set_error("coarse_apply: unknown precision %d", prec);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace coarse
