// Odd-even reduced coarsest system with block-Jacobi left preconditioning (Sec. 2, Sec. 3.2):
//   S v = v - D_ee^{-1} D_eo D_oo^{-1} D_oe v      (v compressed on the even sites),
// applied in factored form by two half applies, each a fused "hops then inverse block" pass
// over the sites of one parity:
//   half(P): u_x = B_x^{-1} g_x,  g_x = z_x - h_x  (or h_x),
//            h_x = sum_mu F_{x,mu} v_{x+mu} + sum_mu sigma3 F_{x-mu,mu}^H sigma3 v_{x-mu}
// (x of parity P, v compressed on the other parity; only the forward hops are stored, the
// backward hop is the neighbour's forward block, as for the full stencil), with the epilogue
// y = u, or y = base - u followed by the polynomial-chain step.  B_x = A_x + i mu sigma3 are
// the diagonal blocks; their inverses are computed once in FP64 (Gauss-Jordan with partial
// pivoting, one CTA per site) and stored per precision.  Each output site reads its 4
// forward blocks, its 4 neighbours' forward blocks and its inverse block: every stored block
// once per half apply, twice per S apply.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "apply_core.cuh"
#include "common.cuh"
#include "batch.cuh"
#include "oddeven.cuh"
#include "pipe.cuh"
#include "tune.cuh"

namespace coarse {
namespace {

// ------------------------------------------------------------------ diagonal-block inverses
// M = [B | I] in shared memory (n x 2n complex double), B = A_x + i mu sigma3; Gauss-Jordan with
// partial pivoting leaves [I | B^{-1}].  A zero pivot marks the site in *bad.
__global__ void __launch_bounds__(256) k_block_inverse(const double2* __restrict__ blocks, int n, double mu,
                                                       double2* __restrict__ inv, int* bad) {
  extern __shared__ double2 M[];  // [n][2n]
  __shared__ double2 fcol[64];
  __shared__ int piv_row;
  const int x = blockIdx.x, n2 = 2 * n;
  const double2* A = blocks + (size_t)x * 5 * n * n;  // self block
  for (int e = threadIdx.x; e < n * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    double2 v = make_double2(0.0, 0.0);
    if (j < n) {
      v = A[(size_t)i * n + j];
      if (i == j) v.y += (i < n / 2 ? mu : -mu);
    } else if (j - n == i) {
      v.x = 1.0;
    }
    M[e] = v;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {  // pivot search over rows k..n-1 of column k by warp 0
      double best = -1.0;
      int row = k;
      for (int i = k + (int)threadIdx.x; i < n; i += 32) {
        const double a = cabs2(M[i * n2 + k]);
        if (a > best) { best = a; row = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int orow = __shfl_xor_sync(0xffffffffu, row, off);
        if (ob > best || (ob == best && orow < row)) { best = ob; row = orow; }
      }
      if (threadIdx.x == 0) piv_row = row;
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k)
      for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        const double2 t = M[k * n2 + j];
        M[k * n2 + j] = M[p * n2 + j];
        M[p * n2 + j] = t;
      }
    __syncthreads();
    const double2 pv = M[k * n2 + k];
    const double pa = cabs2(pv);
    if (pa == 0.0) {
      if (threadIdx.x == 0) atomicExch(bad, 1);
      return;  // uniform: every thread read the same pivot
    }
    const double2 ip = make_double2(pv.x / pa, -pv.y / pa);
    __syncthreads();  // everyone has read M[k][k] before the pivot row is scaled
    for (int j = threadIdx.x; j < n2; j += blockDim.x) M[k * n2 + j] = cmul(M[k * n2 + j], ip);
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = M[i * n2 + k];
    __syncthreads();
    for (int e = threadIdx.x; e < n * n2; e += blockDim.x) {
      const int i = e / n2, j = e % n2;
      if (i == k) continue;
      M[e] = csub(M[e], cmul(fcol[i], M[k * n2 + j]));
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    inv[(size_t)x * n * n + e] = M[i * n2 + n + j];
  }
}

__global__ void k_inv_convert(const double2* __restrict__ in, size_t total, float2* __restrict__ o32,
                              cbf16* __restrict__ o16) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[e];
    if (o32) o32[e] = make_float2((float)v.x, (float)v.y);
    if (o16) {
      cbf16 c;
      c.x = __float2bfloat16_rn((float)v.x);
      c.y = __float2bfloat16_rn((float)v.y);
      o16[e] = c;
    }
  }
}

// ------------------------------------------------------------------------- the half apply
// Block rows from shared memory (the prefetched inverse block).
template <class AC, class BT> struct RowSh;
template <> struct RowSh<double2, double2> {
  template <int CPL> __device__ __forceinline__ static void row(const double2* p, double2 (&e)[CPL]) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) e[c] = p[c];
  }
};
template <> struct RowSh<float2, float2> {
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
template <> struct RowSh<float2, cbf16> {
  template <int CPL> __device__ __forceinline__ static void row(const cbf16* p, float2 (&e)[CPL]) {
    const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      const uint2 v = q[c];
      e[2 * c] = bf2f(v.x);
      e[2 * c + 1] = bf2f(v.y);
    }
  }
};

// One CTA of W warps (W = 4 or 2) per output site x: warp w computes, for its directions
// mu = w, w + W, ..., the forward hop F_{x,mu} v_{x+mu} (row sums) and the backward hop
// sigma3 F_{x-mu,mu}^H sigma3 v_{x-mu} (column sums) into its own slot; h is the sum of the W
// slots in fixed order (deterministic); the inverse block's rows are split over the warps; the
// epilogue runs over the CTA, coalesced.  The site's neighbour record (EoArgs::rec) gives every
// index in one round trip.  PF: thread 0 starts bulk copies of the inverse block and of the
// epilogue's vectors (z, base, acc) into shared memory before the hops, so that nothing after
// the hop sums waits on DRAM; their mbarrier wait is bounded (on expiry: *err raised, the
// copies drained with a second bounded wait, return).  PF needs 16-byte aligned vectors
// (checked by the launcher).
//
// Occupancy: with 2 warps per site and n = 32 in FP32/BF16, 72 registers let 14 CTAs share an SM,
// so that the 2048 sites of one parity of an 8^4 lattice fit in one wave on 152 SMs; the
// prefetching variants are held to that.
template <int N, class AC, int W, bool PF>
constexpr int eo_min_blocks() {
  return (PF && W == 2 && N == 32 && sizeof(decltype(AC{}.x)) == 4) ? 14 : 0;
}
// One output site k of a half apply (the CTA's W warps together); shared by the single-operator
// kernel below and the batched one (one CTA per (solve, site)).
template <int N, class BT, class VT, class AC, int W, bool UNROLL, bool PF>
__device__ __forceinline__ void eo_half_site(const EoArgs& a, const int k) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2, KW = KR / W;  // KW row quads per warp
  constexpr size_t BSZ = (size_t)N * N;
  using AT = decltype(AC{}.x);
  __shared__ AC hpart[W][N];
  __shared__ AC us[N];
  __shared__ __align__(16) BT sinv[PF ? N * N : 1];
  __shared__ __align__(16) VT svec[PF ? 3 * N : 1];  // z, base, acc of this site
  __shared__ __align__(8) uint64_t sbar;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, t = lane & 7;
  const int nh = a.V / 2;
  if (k >= nh) return;  // CTA-uniform
  const int4* rp = a.rec + ((size_t)a.out_par * nh + k) * 4;
  int4 rc[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) rc[mu] = __ldg(rp + mu);
  if (a.stop && *a.stop) return;
  const int x = rc[0].w;
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* v = static_cast<const VT*>(a.v);
  const VT* z = static_cast<const VT*>(a.z);
  const VT* base = static_cast<const VT*>(a.base);
  const bool acc_in = a.mode != APPLY_PLAIN && a.mode != APPLY_POLY_FIRST;
  if constexpr (PF) {
    // the mbarrier is initialised before any thread can wait on it
    if (threadIdx.x == 0) {
      mbar_init(&sbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  if (PF && threadIdx.x == 0) {
    constexpr uint32_t ib = (uint32_t)(BSZ * sizeof(BT)), vb = (uint32_t)(N * sizeof(VT));
    mbar_expect_tx(&sbar, ib + (z ? vb : 0u) + (base ? vb : 0u) + (acc_in ? vb : 0u));
    bulk_g2s(sinv, static_cast<const BT*>(a.inv) + (size_t)x * BSZ, ib, &sbar);
    if (z) bulk_g2s(svec, z + (size_t)k * N, vb, &sbar);
    if (base) bulk_g2s(svec + N, base + (size_t)k * N, vb, &sbar);
    if (acc_in) bulk_g2s(svec + 2 * N, static_cast<const VT*>(a.acc) + (size_t)k * N, vb, &sbar);
  }
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);  // sigma3 of this lane's columns

  AC yf[KR], yb[CPL];
#pragma unroll
  for (int r = 0; r < KR; ++r) yf[r] = AC{0, 0};
#pragma unroll
  for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};
  if (v) {
    // UNROLL: the warp's directions are unrolled so that all their block loads are in flight at once
#pragma unroll (UNROLL ? 4 : 1)
    for (int mu = wid; mu < 4; mu += W) {
      // forward hop: row sums of F_{x,mu} v_{x+mu}; backward: column sums of conj(F_{x-mu,mu}) (sigma3 v)
      const int4 q = mu == 0 ? rc[0] : mu == 1 ? rc[1] : mu == 2 ? rc[2] : rc[3];
      const int fsrc = q.x, nbx = q.y, bsrc = q.z;
      AC w[CPL], xr[KR];
      load_vec<VT, AC, CPL>(v + (size_t)fsrc * N + t * CPL, w);
#pragma unroll
      for (int r = 0; r < KR; ++r) {
        const VT vv = v[(size_t)bsrc * N + 4 * r + g];
        const AT sk = (4 * r + g < NV) ? AT(1) : AT(-1);
        xr[r].x = sk * AT(vv.x);
        xr[r].y = sk * AT(vv.y);
      }
      const BT* fb = B + ((size_t)x * 5 + 1 + mu) * BSZ + g * N + t * CPL;
      const BT* bb = B + ((size_t)nbx * 5 + 1 + mu) * BSZ + g * N + t * CPL;
#pragma unroll
      for (int r = 0; r < KR; ++r) {
        AC e[CPL], f[CPL];
        LoadS<AC, BT>::template row<CPL>(fb + (size_t)r * 4 * N, e);
        LoadS<AC, BT>::template row<CPL>(bb + (size_t)r * 4 * N, f);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          cfma(yf[r], e[c], w[c]);
          cfma_conj(yb[c], f[c], xr[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < KR; ++r)
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      yf[r].x += __shfl_xor_sync(0xffffffffu, yf[r].x, off);
      yf[r].y += __shfl_xor_sync(0xffffffffu, yf[r].y, off);
    }
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int off = 8; off < 32; off <<= 1) {
      yb[c].x += __shfl_xor_sync(0xffffffffu, yb[c].x, off);
      yb[c].y += __shfl_xor_sync(0xffffffffu, yb[c].y, off);
    }
  AC* hp = hpart[wid];
  if (t == 0)
#pragma unroll
    for (int r = 0; r < KR; ++r) hp[4 * r + g] = yf[r];
  __syncwarp();
  if (g == 0)
#pragma unroll
    for (int c = 0; c < CPL; ++c) hp[t * CPL + c] = cadd(hp[t * CPL + c], cscale(yb[c], st));
  if constexpr (PF) {
    // CTA-uniform outcome of the bounded wait for the prefetched inverse and vectors
    if (!__syncthreads_and(mbar_wait(&sbar, 0))) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      mbar_wait(&sbar, 0);  // drain (bounded)
      return;
    }
  } else {
    __syncthreads();
  }
  // g = z - h (or h), h = sum of the 4 direction slots: this lane's column chunk
  AC gi[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = t * CPL + c;
    AC hv = hpart[0][j];
#pragma unroll
    for (int q = 1; q < W; ++q) hv = cadd(hv, hpart[q][j]);
    if (z) {
      const VT zv = PF ? svec[j] : z[(size_t)k * N + j];
      gi[c] = AC{AT(zv.x) - hv.x, AT(zv.y) - hv.y};
    } else {
      gi[c] = hv;
    }
  }
  // u = B_x^{-1} g: warp w takes the row quads w*KW .. w*KW + KW - 1
  {
    AC uf[KW];
#pragma unroll
    for (int q = 0; q < KW; ++q) uf[q] = AC{0, 0};
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      AC e[CPL];
      const size_t off = (size_t)(wid * KW + q) * 4 * N + g * N + t * CPL;
      if constexpr (PF) RowSh<AC, BT>::template row<CPL>(sinv + off, e);
      else LoadS<AC, BT>::template row<CPL>(static_cast<const BT*>(a.inv) + (size_t)x * BSZ + off, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) cfma(uf[q], e[c], gi[c]);
    }
#pragma unroll
    for (int q = 0; q < KW; ++q)
#pragma unroll
      for (int off = 1; off < 8; off <<= 1) {
        uf[q].x += __shfl_xor_sync(0xffffffffu, uf[q].x, off);
        uf[q].y += __shfl_xor_sync(0xffffffffu, uf[q].y, off);
      }
    if (t == 0)
#pragma unroll
      for (int q = 0; q < KW; ++q) us[4 * (wid * KW + q) + g] = uf[q];
  }
  __syncthreads();
  // epilogue over the CTA, coalesced: y = u or base - u, then the chain step with x = base
  VT* y = static_cast<VT*>(a.y);
  const double2 c0d = a.mode != APPLY_PLAIN ? a.coef[0] : make_double2(0.0, 0.0);
  const double2 c1d = a.mode != APPLY_PLAIN ? a.coef[1] : make_double2(0.0, 0.0);
  const double2 c2d = a.mode == APPLY_POLY_FIRST ? a.coef[2] : make_double2(0.0, 0.0);
  const AC c0{AT(c0d.x), AT(c0d.y)}, c1{AT(c1d.x), AT(c1d.y)}, c2{AT(c2d.x), AT(c2d.y)};
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const size_t idx = (size_t)k * N + e;
    AC r = us[e];
    AC xs{0, 0};
    if (base) {
      const VT bv = PF ? svec[N + e] : base[idx];
      xs = AC{AT(bv.x), AT(bv.y)};
      r = csub(xs, r);
    }
    if (a.mode == APPLY_PLAIN) {
      VT o;
      o.x = r.x;
      o.y = r.y;
      y[idx] = o;
    } else {
      // chain step on S: s' = x - c0 (S x) ; acc = acc + c1 s'  (first: acc = c2 x + c1 s')
      VT* accp = static_cast<VT*>(a.acc) + idx;
      AC ac;
      if (a.mode == APPLY_POLY_FIRST) {
        ac = cmul(c2, xs);
      } else {
        const VT av = PF ? svec[2 * N + e] : *accp;
        ac = AC{AT(av.x), AT(av.y)};
      }
      const AC sp = csub(xs, cmul(c0, r));
      ac = cadd(ac, cmul(c1, sp));
      VT o;
      o.x = sp.x;
      o.y = sp.y;
      y[idx] = o;
      VT ao;
      ao.x = ac.x;
      ao.y = ac.y;
      *accp = ao;
    }
  }
}

template <int N, class BT, class VT, class AC, int W, bool UNROLL = false, bool PF = false>
__global__ void __launch_bounds__(32 * W, eo_min_blocks<N, AC, W, PF>()) k_eo_half(EoArgs a) {
  eo_half_site<N, BT, VT, AC, W, UNROLL, PF>(a, blockIdx.x);
}

// Batched half apply: CTA g of the flat grid takes output site g of the n-group (half-site prefix
// sums give its solve), builds that solve's arguments and runs the two-warp unrolled layout.
template <int N, class BT>
__global__ void __launch_bounds__(64) kb_eo_half(BEoApply b) {
  const int g = blockIdx.x;
  if (g >= b.total) return;
  const int k = find_solve(b.site_off, b.count, g);
  const BSolve& s = b.S[b.sidx[k]];
  if (!bgate(s, b.gate)) return;  // uniform for all sites of the solve
  const int step = *b.step;
  EoArgs a{};
  a.blocks = b.poly_blocks ? s.blk_poly : s.blk;
  a.inv = b.poly_blocks ? s.inv_poly : s.inv;
  a.rec = s.eo_rec;
  a.err = s.cnt + s.V;
  a.V = s.V;
  a.out_par = b.out_par;
  a.v = bsel(s, b.vsel, step);
  a.z = bsel(s, b.zsel, step);
  a.base = bsel(s, b.bsel, step);
  a.y = bsel(s, b.ysel, step);
  a.mode = b.mode;
  a.acc = s.acc;
  a.coef = s.polyc + b.coef_off;
  a.stop = nullptr;
  eo_half_site<N, BT, float2, float2, 2, true, false>(a, g - b.site_off[k]);
}

// Warp-per-site variant (4 sites per CTA): one warp walks all 9 blocks of its site.
template <int N, class BT, class VT, class AC>
__global__ void __launch_bounds__(128) k_eo_half_w(EoArgs a) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2;
  constexpr size_t BSZ = (size_t)N * N;
  using AT = decltype(AC{}.x);
  __shared__ AC sh[4][N];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, t = lane & 7;
  const int half = a.V / 2;
  const int k = blockIdx.x * 4 + warp;
  if (k >= half) return;  // warp-uniform
  if (a.stop && *a.stop) return;
  const int4* rp = a.rec + ((size_t)a.out_par * half + k) * 4;
  const int x = __ldg(rp).w;
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* v = static_cast<const VT*>(a.v);
  AC* s = sh[warp];
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);  // sigma3 of this lane's columns

  AC yf[KR], yb[CPL];
#pragma unroll
  for (int r = 0; r < KR; ++r) yf[r] = AC{0, 0};
#pragma unroll
  for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};
  if (v) {
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      // forward hop: row sums of F_{x,mu} v_{x+mu}
      {
        const int src = __ldg(rp + mu).x;
        AC w[CPL];
        load_vec<VT, AC, CPL>(v + (size_t)src * N + t * CPL, w);
        const BT* blk = B + ((size_t)x * 5 + 1 + mu) * BSZ + g * N + t * CPL;
#pragma unroll
        for (int r = 0; r < KR; ++r) {
          AC e[CPL];
          LoadS<AC, BT>::template row<CPL>(blk + (size_t)r * 4 * N, e);
#pragma unroll
          for (int c = 0; c < CPL; ++c) cfma(yf[r], e[c], w[c]);
        }
      }
      // backward hop: column sums of conj(F_{x-mu,mu}) (sigma3 v_{x-mu})
      {
        const int4 q = __ldg(rp + mu);
        const int nbx = q.y, src = q.z;
        AC xr[KR];
#pragma unroll
        for (int r = 0; r < KR; ++r) {
          const VT vv = v[(size_t)src * N + 4 * r + g];
          const AT sk = (4 * r + g < NV) ? AT(1) : AT(-1);
          xr[r].x = sk * AT(vv.x);
          xr[r].y = sk * AT(vv.y);
        }
        const BT* blk = B + ((size_t)nbx * 5 + 1 + mu) * BSZ + g * N + t * CPL;
#pragma unroll
        for (int r = 0; r < KR; ++r) {
          AC e[CPL];
          LoadS<AC, BT>::template row<CPL>(blk + (size_t)r * 4 * N, e);
#pragma unroll
          for (int c = 0; c < CPL; ++c) cfma_conj(yb[c], e[c], xr[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < KR; ++r)
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      yf[r].x += __shfl_xor_sync(0xffffffffu, yf[r].x, off);
      yf[r].y += __shfl_xor_sync(0xffffffffu, yf[r].y, off);
    }
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int off = 8; off < 32; off <<= 1) {
      yb[c].x += __shfl_xor_sync(0xffffffffu, yb[c].x, off);
      yb[c].y += __shfl_xor_sync(0xffffffffu, yb[c].y, off);
    }
  // h = rows (forward) + sigma3-signed columns (backward), assembled in shared memory
  if (t == 0)
#pragma unroll
    for (int r = 0; r < KR; ++r) s[4 * r + g] = yf[r];
  __syncwarp();
  if (g == 0)
#pragma unroll
    for (int c = 0; c < CPL; ++c) s[t * CPL + c] = cadd(s[t * CPL + c], cscale(yb[c], st));
  __syncwarp();
  // g = z - h (or h): this lane's column chunk
  AC gi[CPL];
  const VT* z = static_cast<const VT*>(a.z);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const AC hv = s[t * CPL + c];
    if (z) {
      const VT zv = z[(size_t)k * N + t * CPL + c];
      gi[c] = AC{AT(zv.x) - hv.x, AT(zv.y) - hv.y};
    } else {
      gi[c] = hv;
    }
  }
  // u = B_x^{-1} g: row sums over the inverse block
  AC uf[KR];
#pragma unroll
  for (int r = 0; r < KR; ++r) uf[r] = AC{0, 0};
  {
    const BT* blk = static_cast<const BT*>(a.inv) + (size_t)x * BSZ + g * N + t * CPL;
#pragma unroll
    for (int r = 0; r < KR; ++r) {
      AC e[CPL];
      LoadS<AC, BT>::template row<CPL>(blk + (size_t)r * 4 * N, e);
#pragma unroll
      for (int c = 0; c < CPL; ++c) cfma(uf[r], e[c], gi[c]);
    }
  }
#pragma unroll
  for (int r = 0; r < KR; ++r)
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      uf[r].x += __shfl_xor_sync(0xffffffffu, uf[r].x, off);
      uf[r].y += __shfl_xor_sync(0xffffffffu, uf[r].y, off);
    }
  __syncwarp();  // every lane has read s before it is overwritten
  if (t == 0)
#pragma unroll
    for (int r = 0; r < KR; ++r) s[4 * r + g] = uf[r];
  __syncwarp();
  // epilogue, coalesced: y = u or base - u, then the chain step with x = base
  const VT* base = static_cast<const VT*>(a.base);
  VT* y = static_cast<VT*>(a.y);
  const double2 c0d = a.mode != APPLY_PLAIN ? a.coef[0] : make_double2(0.0, 0.0);
  const double2 c1d = a.mode != APPLY_PLAIN ? a.coef[1] : make_double2(0.0, 0.0);
  const double2 c2d = a.mode == APPLY_POLY_FIRST ? a.coef[2] : make_double2(0.0, 0.0);
  const AC c0{AT(c0d.x), AT(c0d.y)}, c1{AT(c1d.x), AT(c1d.y)}, c2{AT(c2d.x), AT(c2d.y)};
  for (int e = lane; e < N; e += 32) {
    const size_t idx = (size_t)k * N + e;
    AC r = s[e];
    AC xs{0, 0};
    if (base) {
      const VT bv = base[idx];
      xs = AC{AT(bv.x), AT(bv.y)};
      r = csub(xs, r);
    }
    if (a.mode == APPLY_PLAIN) {
      VT o;
      o.x = r.x;
      o.y = r.y;
      y[idx] = o;
    } else {
      // chain step on S: s' = x - c0 (S x) ; acc = acc + c1 s'  (first: acc = c2 x + c1 s')
      VT* accp = static_cast<VT*>(a.acc) + idx;
      AC ac;
      if (a.mode == APPLY_POLY_FIRST) {
        ac = cmul(c2, xs);
      } else {
        const VT av = *accp;
        ac = AC{AT(av.x), AT(av.y)};
      }
      const AC sp = csub(xs, cmul(c0, r));
      ac = cadd(ac, cmul(c1, sp));
      VT o;
      o.x = sp.x;
      o.y = sp.y;
      y[idx] = o;
      VT ao;
      ao.x = ac.x;
      ao.y = ac.y;
      *accp = ao;
    }
  }
}

// ------------------------------------------------------------------ the streamed half apply
// Persistent, warp-specialised variant: one CTA per SM takes a contiguous range of the output
// parity's sites and streams them through a ring of S shared-memory stages.  A stage holds one
// site's operands: its 4 forward blocks (contiguous in memory: one bulk copy), the 4 neighbours'
// forward blocks used as backward hops, its inverse block, the 8 neighbour vectors the hops
// multiply and the epilogue's z, base, acc.  A producer warp reads the sites' neighbour records
// (8 sites per warp-wide load) and issues every copy, completing on the stage's "full" mbarrier,
// as soon as the consumers have released the stage on its "empty" mbarrier.  The 8 consumer
// warps touch no global memory but the output: warp w reduces one hop block (w < 4: F_{x,mu},
// w >= 4: F_{x-mu,mu}, mu = w & 3) against its vector into its slot of hpart; barrier;
// g = z - sum of the 8 slots (fixed order); u = B_x^{-1} g with the inverse's row quads split over
// the warps, the epilogue's operands read into registers; barrier; release; the epilogue as in
// k_eo_half.  The consumers synchronise on named barrier 1 (256 threads) so that the producer
// runs ahead.  The bytes in flight per SM are set by the ring (up to S sites), not by registers.
// Every wait is bounded: an expired consumer wait ends the loop for all consumers (the first
// barrier is a reduction) and raises *err; an expired producer wait stops the producer, which
// then drains its copies still in flight (bounded waits).  Needs v and 16-byte aligned vectors.
constexpr int kEoRingWarps = 8, kEoRingMaxS = 6;
constexpr uint32_t kEoRingThreads = 32 * (kEoRingWarps + 1);

__device__ __forceinline__ int consumers_red_or(int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n barrier.cta.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred), "n"(32 * kEoRingWarps)
      : "memory");
  return r;
}
__device__ __forceinline__ void consumers_sync() {
  asm volatile("barrier.cta.sync 1, %0;" ::"n"(32 * kEoRingWarps) : "memory");
}

// Block-row chunk from shared memory.  For 32-byte chunks (FP32, n = 32) lanes 4..7 of each
// quarter warp take the two 16-byte halves in the opposite order, so that the 8 lanes of a
// 128-bit load phase hit distinct bank groups.
template <class AC, class BT, int CPL>
__device__ __forceinline__ void ring_row(const BT* p, int t, AC (&e)[CPL]) {
  if constexpr (sizeof(BT) == 8 && sizeof(AC) == 8 && CPL == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const int h = (t >> 2) & 1;
    const float4 a = q[h], b = q[h ^ 1];
    const float4 lo = h ? b : a, hi = h ? a : b;
    e[0] = make_float2(lo.x, lo.y);
    e[1] = make_float2(lo.z, lo.w);
    e[2] = make_float2(hi.x, hi.y);
    e[3] = make_float2(hi.z, hi.w);
  } else if constexpr (sizeof(BT) == 4 && (CPL * 4) % 16 == 0) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 4; ++c) {
      const uint4 v = q[c];
      e[4 * c] = bf2f(v.x);
      e[4 * c + 1] = bf2f(v.y);
      e[4 * c + 2] = bf2f(v.z);
      e[4 * c + 3] = bf2f(v.w);
    }
  } else {
    RowSh<AC, BT>::template row<CPL>(p, e);
  }
}

// Shared-memory bytes of one stage of the streamed layout.
template <int N, class BT, class VT>
constexpr size_t eo_ring_stage_bytes() {
  return 9 * (size_t)N * N * sizeof(BT) + 11 * (size_t)N * sizeof(VT);
}

template <int N, class BT, class VT, class AC>
__global__ void __launch_bounds__(kEoRingThreads, 1) k_eo_ring(EoArgs a, int S) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2;
  constexpr size_t BSZ = (size_t)N * N;
  constexpr uint32_t BB = (uint32_t)(BSZ * sizeof(BT)), VB = (uint32_t)(N * sizeof(VT));
  constexpr uint32_t SB = (uint32_t)eo_ring_stage_bytes<N, BT, VT>();
  constexpr uint32_t VO = 9 * BB;  // vector slots: 8 hop vectors (slot = consumer warp), z, base, acc
  using AT = decltype(AC{}.x);
  extern __shared__ __align__(128) unsigned char ring_smem[];
  __shared__ AC hpart[kEoRingWarps][N];
  __shared__ AC us[N];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nh = a.V / 2, G = gridDim.x;
  const int s0 = (int)((long long)nh * blockIdx.x / G), s1 = (int)((long long)nh * (blockIdx.x + 1) / G);
  const int cnt = s1 - s0;  // sites of this CTA (CTA-uniform)
  if (cnt <= 0) return;
  if (a.stop && *a.stop) return;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring_smem + (size_t)S * SB);
  uint64_t* empty = full + S;
  const VT* z = static_cast<const VT*>(a.z);
  const VT* base = static_cast<const VT*>(a.base);
  VT* acc = static_cast<VT*>(a.acc);
  const bool acc_in = a.mode != APPLY_PLAIN && a.mode != APPLY_POLY_FIRST;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (wid == kEoRingWarps) {
    // ---- producer warp
    const int4* R = a.rec + ((size_t)a.out_par * nh + s0) * 4;
    const BT* B = static_cast<const BT*>(a.blocks);
    const BT* INV = static_cast<const BT*>(a.inv);
    const VT* v = static_cast<const VT*>(a.v);
    const uint32_t tx = 9 * BB + 8 * VB + (z ? VB : 0u) + (base ? VB : 0u) + (acc_in ? VB : 0u);
    int issued = 0;
    bool ok = true;
    for (int j0 = 0; j0 < cnt && ok; j0 += 8) {
      // lane l: the record of site j0 + l / 4, direction l % 4
      int4 q = make_int4(0, 0, 0, 0);
      if (j0 + lane / 4 < cnt) q = __ldg(R + (size_t)j0 * 4 + lane);
      for (int jj = 0; jj < 8 && j0 + jj < cnt; ++jj) {
        int4 qm[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          qm[m].x = __shfl_sync(0xffffffffu, q.x, jj * 4 + m);
          qm[m].y = __shfl_sync(0xffffffffu, q.y, jj * 4 + m);
          qm[m].z = __shfl_sync(0xffffffffu, q.z, jj * 4 + m);
          qm[m].w = __shfl_sync(0xffffffffu, q.w, jj * 4 + m);
        }
        const int j = j0 + jj;
        if (lane == 0) {
          // stage j % S is free once the consumers released its previous site j - S
          if (j >= S) ok = mbar_wait(empty + j % S, (uint32_t)((j / S - 1) & 1));
          if (ok) {
            const size_t k = (size_t)s0 + j;
            uint64_t* bar = full + j % S;
            unsigned char* st = ring_smem + (size_t)(j % S) * SB;
            const size_t x = (size_t)qm[0].w;
            mbar_expect_tx(bar, tx);
            bulk_g2s(st, B + (x * 5 + 1) * BSZ, 4 * BB, bar);
#pragma unroll
            for (int m = 0; m < 4; ++m)
              bulk_g2s(st + (4 + m) * BB, B + ((size_t)qm[m].y * 5 + 1 + m) * BSZ, BB, bar);
            bulk_g2s(st + 8 * BB, INV + x * BSZ, BB, bar);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              bulk_g2s(st + VO + m * VB, v + (size_t)qm[m].x * N, VB, bar);
              bulk_g2s(st + VO + (4 + m) * VB, v + (size_t)qm[m].z * N, VB, bar);
            }
            if (z) bulk_g2s(st + VO + 8 * VB, z + k * N, VB, bar);
            if (base) bulk_g2s(st + VO + 9 * VB, base + k * N, VB, bar);
            if (acc_in) bulk_g2s(st + VO + 10 * VB, acc + k * N, VB, bar);
            ++issued;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
    }
    if (!ok && lane == 0) atomicExch(a.err, 1);
    // The copies of the last stages issued must have landed before the CTA exits, also when every
    // copy was issued and the consumers then stopped on a timeout of their own: wait (bounded) on
    // their full barriers.  After a normal run these phases are complete and the waits return at once.
    if (lane == 0)
      for (int j = max(0, issued - S); j < issued; ++j) mbar_wait(full + j % S, (uint32_t)((j / S) & 1));
    return;
  }

  // ---- consumer warps
  const int g = lane >> 3, t = lane & 7;
  const bool bwd = wid >= 4;
  const AT st = (t * CPL < NV) ? AT(1) : AT(-1);  // sigma3 of this lane's columns
  const double2 c0d = a.mode != APPLY_PLAIN ? a.coef[0] : make_double2(0.0, 0.0);
  const double2 c1d = a.mode != APPLY_PLAIN ? a.coef[1] : make_double2(0.0, 0.0);
  const double2 c2d = a.mode == APPLY_POLY_FIRST ? a.coef[2] : make_double2(0.0, 0.0);
  const AC c0{AT(c0d.x), AT(c0d.y)}, c1{AT(c1d.x), AT(c1d.y)}, c2{AT(c2d.x), AT(c2d.y)};
  VT* y = static_cast<VT*>(a.y);
  const int ne = threadIdx.x;  // epilogue element of this thread (if < N)
  for (int i = 0; i < cnt; ++i) {
    const size_t k = (size_t)s0 + i;
    // warp-uniform outcome (the shuffles below need the whole warp)
    const bool ok = __all_sync(0xffffffffu, mbar_wait(full + i % S, (uint32_t)((i / S) & 1)));
    const unsigned char* sp = ring_smem + (size_t)(i % S) * SB;
    if (ok) {
      const BT* blk = reinterpret_cast<const BT*>(sp + (size_t)wid * BB) + g * N + t * CPL;
      const VT* vec = reinterpret_cast<const VT*>(sp + VO + (size_t)wid * VB);
      if (!bwd) {
        // row sums of F_{x,mu} v_{x+mu}
        AC w[CPL], yf[KR];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const VT e = vec[t * CPL + c];
          w[c] = AC{AT(e.x), AT(e.y)};
        }
#pragma unroll
        for (int r = 0; r < KR; ++r) {
          AC e[CPL];
          ring_row<AC, BT, CPL>(blk + (size_t)r * 4 * N, t, e);
          yf[r] = AC{0, 0};
#pragma unroll
          for (int c = 0; c < CPL; ++c) cfma(yf[r], e[c], w[c]);
        }
#pragma unroll
        for (int r = 0; r < KR; ++r)
#pragma unroll
          for (int off = 1; off < 8; off <<= 1) {
            yf[r].x += __shfl_xor_sync(0xffffffffu, yf[r].x, off);
            yf[r].y += __shfl_xor_sync(0xffffffffu, yf[r].y, off);
          }
        if (t == 0)
#pragma unroll
          for (int r = 0; r < KR; ++r) hpart[wid][4 * r + g] = yf[r];
      } else {
        // column sums of conj(F_{x-mu,mu}) (sigma3 v_{x-mu}), then sigma3 on the result
        AC yb[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) yb[c] = AC{0, 0};
#pragma unroll
        for (int r = 0; r < KR; ++r) {
          const VT e = vec[4 * r + g];
          const AT sk = (4 * r + g < NV) ? AT(1) : AT(-1);
          const AC xr{sk * AT(e.x), sk * AT(e.y)};
          AC f[CPL];
          ring_row<AC, BT, CPL>(blk + (size_t)r * 4 * N, t, f);
#pragma unroll
          for (int c = 0; c < CPL; ++c) cfma_conj(yb[c], f[c], xr);
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int off = 8; off < 32; off <<= 1) {
            yb[c].x += __shfl_xor_sync(0xffffffffu, yb[c].x, off);
            yb[c].y += __shfl_xor_sync(0xffffffffu, yb[c].y, off);
          }
        if (g == 0)
#pragma unroll
          for (int c = 0; c < CPL; ++c) hpart[wid][t * CPL + c] = cscale(yb[c], st);
      }
    }
    if (consumers_red_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;  // all consumers; the producer drains its copies
    }
    AC bv{0, 0}, av{0, 0};
    {
      const VT* sv = reinterpret_cast<const VT*>(sp + VO + 8 * (size_t)VB);  // z, base, acc
      AC gi[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = t * CPL + c;
        AC hv = hpart[0][j];
#pragma unroll
        for (int w = 1; w < kEoRingWarps; ++w) hv = cadd(hv, hpart[w][j]);
        if (z) {
          const VT e = sv[j];
          gi[c] = AC{AT(e.x) - hv.x, AT(e.y) - hv.y};
        } else {
          gi[c] = hv;
        }
      }
      const BT* iblk = reinterpret_cast<const BT*>(sp + 8 * (size_t)BB) + g * N + t * CPL;
      for (int q = wid; q < KR; q += kEoRingWarps) {
        AC e[CPL];
        ring_row<AC, BT, CPL>(iblk + (size_t)q * 4 * N, t, e);
        AC uf{0, 0};
#pragma unroll
        for (int c = 0; c < CPL; ++c) cfma(uf, e[c], gi[c]);
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
          uf.x += __shfl_xor_sync(0xffffffffu, uf.x, off);
          uf.y += __shfl_xor_sync(0xffffffffu, uf.y, off);
        }
        if (t == 0) us[4 * q + g] = uf;
      }
      if (ne < N) {
        if (base) {
          const VT e = sv[N + ne];
          bv = AC{AT(e.x), AT(e.y)};
        }
        if (acc_in) {
          const VT e = sv[2 * N + ne];
          av = AC{AT(e.x), AT(e.y)};
        }
      }
    }
    consumers_sync();
    // every consumer is done with the stage: release it to the producer
    if (threadIdx.x == 0) mbar_arrive(empty + i % S);
    if (ne < N) {
      const size_t idx = k * N + ne;
      AC r = us[ne];
      if (base) r = csub(bv, r);
      if (a.mode == APPLY_PLAIN) {
        VT o;
        o.x = r.x;
        o.y = r.y;
        y[idx] = o;
      } else {
        // chain step on S: s' = x - c0 (S x) ; acc = acc + c1 s'  (first: acc = c2 x + c1 s')
        AC acv = a.mode == APPLY_POLY_FIRST ? cmul(c2, bv) : av;
        const AC spv = csub(bv, cmul(c0, r));
        acv = cadd(acv, cmul(c1, spv));
        VT o;
        o.x = spv.x;
        o.y = spv.y;
        y[idx] = o;
        VT ao;
        ao.x = acv.x;
        ao.y = acv.y;
        acc[idx] = ao;
      }
    }
  }
}

// full vector <-> (even, odd) compressed halves
template <class VT>
__global__ void k_eo_split(const VT* __restrict__ full, const int* __restrict__ sites, int V, int n, VT* ev, VT* od) {
  const int half = V / 2;
  const size_t total = (size_t)V * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / n), e = (int)(i % n);  // q-th site of the (even, odd) list
    const int x = __ldg(sites + q);
    VT* dst = q < half ? ev : od;
    dst[(size_t)(q < half ? q : q - half) * n + e] = full[(size_t)x * n + e];
  }
}
template <class VT>
__global__ void k_eo_merge(const VT* __restrict__ ev, const VT* __restrict__ od, const int* __restrict__ sites, int V,
                           int n, VT* full) {
  const int half = V / 2;
  const size_t total = (size_t)V * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / n), e = (int)(i % n);
    const int x = __ldg(sites + q);
    const VT* src = q < half ? ev : od;
    full[(size_t)x * n + e] = src[(size_t)(q < half ? q : q - half) * n + e];
  }
}

int grid_of(size_t total) {
  size_t g = (total + 255) / 256;
  const size_t cap = (size_t)sm_count() * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int eo_prepare(coarse_op* op, double mu_eff, cudaStream_t s) {
  if (!op->eo_sites) {
    set_error("odd-even reduction needs even lattice extents (got %d x %d x %d x %d)", op->dims[0], op->dims[1],
              op->dims[2], op->dims[3]);
    return COARSE_ERR_INVALID_ARG;
  }
  // inverses per mass sign (+mu: D_c, -mu: the adjoint system's D_c(-mu)); mu = 0 has one set
  const int sg = eo_sign(op, mu_eff);
  if (op->inv_ok[sg]) return COARSE_OK;
  const int n = op->n;
  const size_t nn = (size_t)op->V * n * n;
  const size_t esz[3] = {sizeof(double2), sizeof(float2), sizeof(cbf16)};
  for (int p = 0; p < 3; ++p) {
    if (!op->blk[p].ptr || op->inv[sg][p].ptr) continue;
    op->inv[sg][p].bytes = nn * esz[p];
    if (cudaMalloc(&op->inv[sg][p].ptr, op->inv[sg][p].bytes) != cudaSuccess) {
      cudaGetLastError();
      op->inv[sg][p].ptr = nullptr;
      set_error("odd-even: allocation of the block inverses failed");
      return COARSE_ERR_OOM;
    }
  }
  const size_t smem = sizeof(double2) * (size_t)n * 2 * n;
  static bool attr = false;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr = true;
  }
  COARSE_CUDA(cudaMemsetAsync(op->apply_cnt + op->V + 1, 0, sizeof(int), s));
  k_block_inverse<<<op->V, 256, smem, s>>>((const double2*)op->blk[0].ptr, n, mu_eff, (double2*)op->inv[sg][0].ptr,
                                           op->apply_cnt + op->V + 1);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  k_inv_convert<<<grid_of(nn), 256, 0, s>>>((const double2*)op->inv[sg][0].ptr, nn, (float2*)op->inv[sg][1].ptr,
                                             (cbf16*)op->inv[sg][2].ptr);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  int bad = 0;
  COARSE_CUDA(cudaMemcpyAsync(&bad, op->apply_cnt + op->V + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  COARSE_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    set_error("odd-even: a diagonal block A_x + i mu sigma3 is singular");
    return COARSE_ERR_NONFINITE;
  }
  op->inv_ok[sg] = 1;
  return COARSE_OK;
}

namespace {

// The streamed layout: S stages of one site's operands, as many as fit (at most kEoRingMaxS); one
// CTA per SM.  INVALID_ARG if not even one stage fits.
template <int N, class BT, class VT, class AC>
int launch_eo_ring_n(const EoArgs& a, cudaStream_t s) {
  constexpr size_t SB = eo_ring_stage_bytes<N, BT, VT>();
  static int S = -1;
  static size_t dyn = 0;
  if (S < 0) {
    int dev = 0, optin = 0;
    COARSE_CUDA(cudaGetDevice(&dev));
    COARSE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    COARSE_CUDA(cudaFuncGetAttributes(&fa, k_eo_ring<N, BT, VT, AC>));
    // the ring and its mbarriers, next to the static shared memory and the dynamic part's alignment
    int sv = kEoRingMaxS;
    for (; sv >= 1; --sv) {
      dyn = (size_t)sv * SB + 16 * (size_t)sv;
      if (dyn + fa.sharedSizeBytes + 128 <= (size_t)optin) break;
    }
    if (sv >= 1)
      COARSE_CUDA(cudaFuncSetAttribute(k_eo_ring<N, BT, VT, AC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dyn));
    S = std::max(sv, 0);
  }
  if (S < 1) {
    set_error("odd-even: the streamed layout does not fit in shared memory for n = %d", N);
    return COARSE_ERR_INVALID_ARG;
  }
  const int grid = std::min(a.V / 2, sm_count());
  k_eo_ring<N, BT, VT, AC><<<grid, kEoRingThreads, dyn, s>>>(a, S);
  return COARSE_OK;
}

template <class BT, class VT, class AC>
int launch_eo_variant(int variant, int n, const EoArgs& a, cudaStream_t s) {
  const int half = a.V / 2;
  // the prefetching and streamed variants copy vectors with bulk copies: 16-byte aligned only
  const uintptr_t al = (uintptr_t)a.z | (uintptr_t)a.base | (uintptr_t)a.acc | (uintptr_t)a.inv;
  if (variant == 6) {
    if constexpr (sizeof(decltype(AC{}.x)) == 4) {
      if (a.v && !((al | (uintptr_t)a.v) & 15)) {
        int rc = COARSE_ERR_INVALID_ARG;
        switch (n) {
          case 16: rc = launch_eo_ring_n<16, BT, VT, AC>(a, s); break;
          case 32: rc = launch_eo_ring_n<32, BT, VT, AC>(a, s); break;
          case 48: rc = launch_eo_ring_n<48, BT, VT, AC>(a, s); break;
          default: set_error("odd-even: unsupported n = %d", n);
        }
        if (rc != COARSE_OK) return rc;
        note_launch();
        COARSE_CUDA(cudaGetLastError());
        return COARSE_OK;
      }
    }
    variant = 4;  // FP64 blocks, no hop input (the right-hand side pass) or unaligned vectors
  }
  if (variant >= 4 && (al & 15)) variant -= 2;
#define EO_LAUNCH(NN)                                                                           \
  case NN:                                                                                      \
    if (variant == 1) k_eo_half_w<NN, BT, VT, AC><<<(half + 3) / 4, 128, 0, s>>>(a);             \
    else if (variant == 2) k_eo_half<NN, BT, VT, AC, 2><<<half, 64, 0, s>>>(a);                  \
    else if (variant == 3) k_eo_half<NN, BT, VT, AC, 2, true><<<half, 64, 0, s>>>(a);            \
    else if (variant == 4) k_eo_half<NN, BT, VT, AC, 2, false, true><<<half, 64, 0, s>>>(a);     \
    else if (variant == 5) k_eo_half<NN, BT, VT, AC, 2, true, true><<<half, 64, 0, s>>>(a);      \
    else k_eo_half<NN, BT, VT, AC, 4><<<half, 128, 0, s>>>(a);                                   \
    break;
  switch (n) {
    EO_LAUNCH(16)
    EO_LAUNCH(32)
    EO_LAUNCH(48)
    default: set_error("odd-even: unsupported n = %d", n); return COARSE_ERR_INVALID_ARG;
  }
#undef EO_LAUNCH
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

// The autotuner picks, per (precision, n, lattice-size bucket), between one CTA of 4 warps per
// site (candidate 0), one warp per site (candidate 1) and one CTA of 2 warps per site with the
// direction loop rolled (candidates 2, 4) or unrolled (3, 5), the last two with the inverse block
// and the epilogue vectors prefetched into shared memory, and (FP32 / BF16 blocks) the streamed
// persistent layout (6); candidates run in plain mode into a scratch output.
template <class BT, class VT, class AC>
int launch_eo_tuned(int prec, int n, const EoArgs& a, cudaStream_t s) {
  const int ni = n / 16 - 1, vb = std::min(tune_bucket(a.V), 31);
  if (ni < 0 || ni > 2) {
    set_error("odd-even: unsupported n = %d", n);
    return COARSE_ERR_INVALID_ARG;
  }
  int choice = tune_fast_get(1, prec, ni, vb);
  if (choice < 0) {
    char key[64];
    snprintf(key, sizeof(key), "eo/p%d/n%d/v%d", prec, n, vb);
    void* scratch = nullptr;
    const size_t hv = (size_t)(a.V / 2) * n;
    auto run = [&](const TuneChoice& c) -> int {
      if (!scratch) {
        if (cudaMalloc(&scratch, 2 * sizeof(VT) * hv) != cudaSuccess) {
          cudaGetLastError();
          scratch = nullptr;
          set_error("odd-even: autotuner scratch allocation failed");
          return COARSE_ERR_OOM;
        }
        COARSE_CUDA(cudaMemsetAsync(scratch, 0, 2 * sizeof(VT) * hv, s));
      }
      EoArgs t = a;
      // candidates are always timed with the hops (a pass without them is not representative)
      if (!t.v) t.v = static_cast<VT*>(scratch) + hv;
      t.mode = APPLY_PLAIN;
      t.y = scratch;
      t.acc = nullptr;
      t.coef = nullptr;
      t.stop = nullptr;
      return launch_eo_variant<BT, VT, AC>(c.a, n, t, s);
    };
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    TuneChoice c;
    std::vector<TuneChoice> cands;
    for (int v = 0; v <= 6; ++v)
      if (v < 6 || sizeof(decltype(AC{}.x)) == 4) cands.push_back(TuneChoice{v, 0, 0});
    const int rc = tune_pick(key, cands, run, s, &c);
    if (scratch) {
      cudaStreamSynchronize(s);
      cudaFree(scratch);
    }
    if (rc != COARSE_OK) return rc;
    if (cap == cudaStreamCaptureStatusNone) tune_fast_put(1, prec, ni, vb, c.a);
    choice = c.a;
  }
  return launch_eo_variant<BT, VT, AC>(choice, n, a, s);
}

}  // namespace

int launch_eo_half(int prec, int n, const EoArgs& a, cudaStream_t s) {
  if (a.V / 2 <= 0) return COARSE_OK;
  switch (prec) {
    case COARSE_PREC_FP64: return launch_eo_tuned<double2, double2, double2>(prec, n, a, s);
    case COARSE_PREC_FP32: return launch_eo_tuned<float2, float2, float2>(prec, n, a, s);
    case COARSE_PREC_BF16: return launch_eo_tuned<cbf16, float2, float2>(prec, n, a, s);
  }
  set_error("odd-even: unknown precision %d", prec);
  return COARSE_ERR_INVALID_ARG;
}

int launch_eo_split(int v64, const void* full, const int* sites, int V, int n, void* ev, void* od, cudaStream_t s) {
  const size_t total = (size_t)V * n;
  if (v64) k_eo_split<double2><<<grid_of(total), 256, 0, s>>>((const double2*)full, sites, V, n, (double2*)ev, (double2*)od);
  else k_eo_split<float2><<<grid_of(total), 256, 0, s>>>((const float2*)full, sites, V, n, (float2*)ev, (float2*)od);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_eo_merge(int v64, const void* ev, const void* od, const int* sites, int V, int n, void* full, cudaStream_t s) {
  const size_t total = (size_t)V * n;
  if (v64) k_eo_merge<double2><<<grid_of(total), 256, 0, s>>>((const double2*)ev, (const double2*)od, sites, V, n, (double2*)full);
  else k_eo_merge<float2><<<grid_of(total), 256, 0, s>>>((const float2*)ev, (const float2*)od, sites, V, n, (float2*)full);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

// y = S x on compressed even vectors (t: odd scratch of the vector type), with an optional
// polynomial-chain epilogue (mode, acc, coef) as the full stencil's.
int launch_beo_half(int prec, int n, const BEoApply& b, cudaStream_t s) {
  if (b.total <= 0) return COARSE_OK;
  const dim3 grid(b.total);
#define BEO(NN)                                                                              \
  if (prec == COARSE_PREC_BF16) kb_eo_half<NN, cbf16><<<grid, 64, 0, s>>>(b);                \
  else kb_eo_half<NN, float2><<<grid, 64, 0, s>>>(b);
  switch (n) {
    case 16: BEO(16) break;
    case 32: BEO(32) break;
    case 48: BEO(48) break;
    default: set_error("batched odd-even: unsupported n = %d", n); return COARSE_ERR_INVALID_ARG;
  }
#undef BEO
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_eo_schur(const coarse_op* op, int prec, double mu_eff, const void* x, void* y, void* t, int mode, void* acc,
                    const double2* coef, const int* stop, cudaStream_t s) {
  EoArgs a{};
  a.blocks = op->blk[prec].ptr;
  a.inv = op->inv[eo_sign(op, mu_eff)][prec].ptr;
  a.rec = op->eo_rec;
  a.err = op->apply_cnt + op->V;
  a.V = op->V;
  a.stop = stop;
  // t_o = D_oo^{-1} D_oe x
  a.out_par = 1;
  a.v = x;
  a.z = nullptr;
  a.base = nullptr;
  a.y = t;
  a.mode = APPLY_PLAIN;
  a.acc = nullptr;
  a.coef = nullptr;
  int rc = launch_eo_half(prec, op->n, a, s);
  if (rc != COARSE_OK) return rc;
  // y = x - D_ee^{-1} D_eo t_o (then the chain step)
  a.out_par = 0;
  a.v = t;
  a.base = x;
  a.y = y;
  a.mode = mode;
  a.acc = acc;
  a.coef = coef;
  return launch_eo_half(prec, op->n, a, s);
}

}  // namespace coarse
