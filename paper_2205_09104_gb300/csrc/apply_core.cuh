// Per-site body of the coarse stencil apply (shared by the single-operator and the batched
// kernels): loads, the push-pull site computation and the site finisher.
#pragma once

#include "common.cuh"

namespace coarse {

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

// Block loads (each block entry is read once per pass): plain non-coherent loads.  The
// evict-first hint (ld.global.cs) was measured slower on every stencil and half apply at 16^4,
// n = 48 (FP32 S apply 1883-2366 us vs 1594-1614 us, BF16 904-916 vs 833-852, full FP32
// stencil 1152 vs 969), the more so after any other kernel had touched memory, while DRAM
// traffic stayed at the algorithmic bytes either way.
template <class T> __device__ __forceinline__ T ld_stream(const T* p) { return __ldg(p); }

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
// One warp processes site `site` of the launch described by `a` (ys_w: n accumulator entries
// of shared memory owned by the warp).
template <int N, class BT, class VT, class AC>
__device__ __forceinline__ void apply_site(const ApplyArgs& a, int site, AC* ys_w) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2;
  using AT = decltype(AC{}.x);
  const int lane = threadIdx.x & 31;
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
      ys_w[4 * k + g] = cscale(yf[k], sr);
    }
  }
  __syncwarp();
  if (g == 0) {
    AC* dst = Pb + (size_t)site * N + t * CPL;
#pragma unroll
    for (int c = 0; c < CPL; ++c) dst[c] = ys_w[t * CPL + c];
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


}  // namespace coarse
