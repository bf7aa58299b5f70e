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
#include "oddeven.cuh"
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
// One CTA of W warps (W = 4 or 2) per output site x: warp w computes, for its directions
// mu = w, w + W, ..., the forward hop F_{x,mu} v_{x+mu} (row sums) and the backward hop
// sigma3 F_{x-mu,mu}^H sigma3 v_{x-mu} (column sums) into its own slot; h is the sum of the W
// slots in fixed order (deterministic); the inverse block's rows are split over the warps; the
// epilogue runs over the CTA, coalesced.
template <int N, class BT, class VT, class AC, int W, bool UNROLL = false>
__global__ void __launch_bounds__(32 * W) k_eo_half(EoArgs a) {
  constexpr int CPL = N / 8, KR = N / 4, NV = N / 2, KW = KR / W;  // KW row quads per warp
  constexpr size_t BSZ = (size_t)N * N;
  using AT = decltype(AC{}.x);
  __shared__ AC hpart[W][N];
  __shared__ AC us[N];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, t = lane & 7;
  const int k = blockIdx.x;
  if (k >= a.V / 2) return;  // CTA-uniform
  if (a.stop && *a.stop) return;
  const int x = __ldg(a.sites + a.out_par * (a.V / 2) + k);
  const BT* B = static_cast<const BT*>(a.blocks);
  const VT* v = static_cast<const VT*>(a.v);
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
      const int fsrc = __ldg(a.half + __ldg(a.nb + x * 8 + mu));
      const int nbx = __ldg(a.nb + x * 8 + 4 + mu);
      const int bsrc = __ldg(a.half + nbx);
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
  __syncthreads();
  // g = z - h (or h), h = sum of the 4 direction slots: this lane's column chunk
  AC gi[CPL];
  const VT* z = static_cast<const VT*>(a.z);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = t * CPL + c;
    AC hv = hpart[0][j];
#pragma unroll
    for (int q = 1; q < W; ++q) hv = cadd(hv, hpart[q][j]);
    if (z) {
      const VT zv = z[(size_t)k * N + j];
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
    const BT* blk = static_cast<const BT*>(a.inv) + (size_t)x * BSZ + g * N + t * CPL;
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      AC e[CPL];
      LoadS<AC, BT>::template row<CPL>(blk + (size_t)(wid * KW + q) * 4 * N, e);
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
  const VT* base = static_cast<const VT*>(a.base);
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
  const int x = __ldg(a.sites + a.out_par * half + k);
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
        const int src = __ldg(a.half + __ldg(a.nb + x * 8 + mu));
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
        const int nbx = __ldg(a.nb + x * 8 + 4 + mu);
        const int src = __ldg(a.half + nbx);
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

template <class BT, class VT, class AC>
int launch_eo_variant(int variant, int n, const EoArgs& a, cudaStream_t s) {
  const int half = a.V / 2;
#define EO_LAUNCH(NN)                                                                           \
  case NN:                                                                                      \
    if (variant == 1) k_eo_half_w<NN, BT, VT, AC><<<(half + 3) / 4, 128, 0, s>>>(a);             \
    else if (variant == 2) k_eo_half<NN, BT, VT, AC, 2><<<half, 64, 0, s>>>(a);                  \
    else if (variant == 3) k_eo_half<NN, BT, VT, AC, 2, true><<<half, 64, 0, s>>>(a);            \
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
// direction loop rolled (candidate 2) or unrolled (candidate 3); candidates run in plain mode into
// a scratch output.
template <class BT, class VT, class AC>
int launch_eo_tuned(int prec, int n, const EoArgs& a, cudaStream_t s) {
  static int choice[3][32];
  static bool init = false;
  if (!init) {
    for (auto& row : choice)
      for (int& c : row) c = -1;
    init = true;
  }
  const int ni = n / 16 - 1, vb = std::min(tune_bucket(a.V), 31);
  if (ni < 0 || ni > 2) {
    set_error("odd-even: unsupported n = %d", n);
    return COARSE_ERR_INVALID_ARG;
  }
  if (choice[ni][vb] < 0) {
    char key[64];
    snprintf(key, sizeof(key), "eo/p%d/n%d/v%d", prec, n, vb);
    void* scratch = nullptr;
    auto run = [&](const TuneChoice& c) -> int {
      if (!scratch && cudaMalloc(&scratch, sizeof(VT) * (size_t)(a.V / 2) * n) != cudaSuccess) {
        cudaGetLastError();
        set_error("odd-even: autotuner scratch allocation failed");
        return COARSE_ERR_OOM;
      }
      EoArgs t = a;
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
    const int rc = tune_pick(key, {TuneChoice{0, 0, 0}, TuneChoice{1, 0, 0}, TuneChoice{2, 0, 0}, TuneChoice{3, 0, 0}},
                             run, s, &c);
    if (scratch) {
      cudaStreamSynchronize(s);
      cudaFree(scratch);
    }
    if (rc != COARSE_OK) return rc;
    if (cap != cudaStreamCaptureStatusNone) return launch_eo_variant<BT, VT, AC>(c.a, n, a, s);
    choice[ni][vb] = c.a;
  }
  return launch_eo_variant<BT, VT, AC>(choice[ni][vb], n, a, s);
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
int launch_eo_schur(const coarse_op* op, int prec, double mu_eff, const void* x, void* y, void* t, int mode, void* acc,
                    const double2* coef, const int* stop, cudaStream_t s) {
  EoArgs a{};
  a.blocks = op->blk[prec].ptr;
  a.inv = op->inv[eo_sign(op, mu_eff)][prec].ptr;
  a.nb = op->nb;
  a.sites = op->eo_sites;
  a.half = op->eo_half;
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
