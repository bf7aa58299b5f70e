// Multi-right-hand-side stencil on tensor cores: Y = D_c X for up to 12 columns per pass with
// BF16 blocks, BF16 vector fragments and FP32 accumulation (mma.sync m16n8k16).
//
// Per site x this is the GEMM [n x 9n] . [9n x R] of Eq. (6): the self block, the four forward
// blocks F_{x,mu} and the four backward blocks sigma3 F_{x-mu,mu}^H sigma3 (Sec. 4.2's storage of
// only the forward hops), applied to the gathered vectors of the 9 sites.
//
// Complex as real.  Block F = Fr + i Fi gives two real A operands Fr, Fi.  Four columns q of a
// column tile give the real B operand X~[k][2q + c] = (c == 0 ? Re : Im) x_q[k].  Then
//   P1 = Fr X~, P2 = Fi X~:   (F x_q)_a   = (P1[a][2q] - P2[a][2q+1], P1[a][2q+1] + P2[a][2q])
//   Q1 = Fr^T X~, Q2 = Fi^T X~: (F^H x_q)_j = (Q1[j][2q] + Q2[j][2q+1], Q1[j][2q+1] - Q2[j][2q])
// so every complex multiply-add is 4 real ones, as on CUDA cores.
//
// Fragment-native block layout (built once from the BF16 blocks by k_pack_mrhs):
//   word index ((((x*5 + b)*NT + ti)*NT + tk)*2 + p)*128 + lane*4 + w,   NT = n/16,
//   lane = 4g + t, word w holds plane p (0 re, 1 im) of F[16ti + g + 8(w&1)][16tk + 2t + 8(w>>1) + {0,1}]
// which is exactly the lane's m16n8k16 A fragment {a0, a1, a2, a3} of tile (ti, tk): one 16-byte
// coalesced load per lane per tile and plane.  The transpose F^T of a tile is made in registers
// with movmatrix (a0' = T(a0), a1' = T(a2), a2' = T(a1), a3' = T(a3)).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace coarse {

constexpr int kMrhsTile = 4;    // columns per tensor-core tile (B operand is 8 wide: re, im of 4 columns)
constexpr int kMrhsMaxT = 3;    // tiles per pass: up to 12 columns

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t movmatrix_t(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(d) : "r"(a));
  return d;
}

// fragment of the transposed 16x16 tile
__device__ __forceinline__ uint4 frag_transpose(const uint4& a) {
  return make_uint4(movmatrix_t(a.x), movmatrix_t(a.z), movmatrix_t(a.y), movmatrix_t(a.w));
}

__device__ __forceinline__ uint32_t bf2_bits(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Where the columns of one pass live: column q of the pass is x + q * ldx (complex64 elements).
struct MrhsCols {
  const float2* x;
  float2* y;
  long long ldx, ldy;
  int R;  // columns in this pass (1..12)
};

// B fragments of vector site s, k tile kt, column tile tl: lane (g, t) feeds column 4tl + g/2,
// real (g even) or imaginary (g odd) part, of entries 16kt + 2t + {0, 1} (b0) and + 8 (b1).
// neg_lo / neg_hi: flip the sign of the entries of the first / second half of the k tile.
template <int N>
__device__ __forceinline__ void mrhs_bfrag(const MrhsCols& c, int s, int kt, int tl, uint32_t neg_lo,
                                           uint32_t neg_hi, uint32_t& b0, uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int q = kMrhsTile * tl + (g >> 1);
  if (q >= c.R) { b0 = b1 = 0u; return; }
  const float4* p = reinterpret_cast<const float4*>(c.x + q * c.ldx + (size_t)s * N + 16 * kt + 2 * t);
  const float4 lo = __ldg(p), hi = __ldg(p + 4);
  b0 = ((g & 1) ? bf2_bits(lo.y, lo.w) : bf2_bits(lo.x, lo.z)) ^ neg_lo;
  b1 = ((g & 1) ? bf2_bits(hi.y, hi.w) : bf2_bits(hi.x, hi.z)) ^ neg_hi;
}

// One warp computes output rows 16rt .. 16rt+15 of site x for all columns of the pass.
//   y_q[x] = o (P + s3 Q + i mu' v),  P = A_x w_x + sum_mu F_{x,mu} w_{x+mu},
//   Q = sum_mu F_{x-mu,mu}^H (s3 w_{x-mu}),  w = (adj ? s3 x : x),  v = (adj ? x : s3 x),
//   o = (adj ? s3 : 1), mu' = adj ? -mu : mu (passed in already signed).
// adj = 1 gives D^H = s3 D(-mu) s3 (gamma5-hermiticity, Sec. 2).
template <int N, int T>
__device__ __forceinline__ void mrhs_rows(const uint4* __restrict__ frag, const int* __restrict__ nb,
                                          const MrhsCols& c, int x, int rt, float mu, int adj) {
  constexpr int NT = N / 16, NV = N / 2;
  constexpr size_t TILE = 2 * 32;  // uint4 per tile (two planes)
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float P1[T][4], P2[T][4], Q1[T][4], Q2[T][4];
#pragma unroll
  for (int tl = 0; tl < T; ++tl)
#pragma unroll
    for (int i = 0; i < 4; ++i) P1[tl][i] = P2[tl][i] = Q1[tl][i] = Q2[tl][i] = 0.f;
  // sign masks of sigma3 per half k tile (NV is a multiple of 8, so uniform over the warp)
  auto s3mask = [](int k0) -> uint32_t { return k0 < NV ? 0u : 0x80008000u; };

  // ---- pull: self block and forward hops
#pragma unroll 1
  for (int b = 0; b < 5; ++b) {
    const int s = b == 0 ? x : __ldg(nb + x * 8 + (b - 1));
    const uint4* base = frag + (((size_t)x * 5 + b) * NT + rt) * NT * TILE;
#pragma unroll
    for (int kt = 0; kt < NT; ++kt) {
      const uint4 are = __ldg(base + kt * TILE + lane);
      const uint4 aim = __ldg(base + kt * TILE + 32 + lane);
      const uint32_t nl = adj ? s3mask(16 * kt) : 0u, nh = adj ? s3mask(16 * kt + 8) : 0u;
#pragma unroll
      for (int tl = 0; tl < T; ++tl) {
        uint32_t b0, b1;
        mrhs_bfrag<N>(c, s, kt, tl, nl, nh, b0, b1);
        mma_bf16(P1[tl], are, b0, b1);
        mma_bf16(P2[tl], aim, b0, b1);
      }
    }
  }
  // ---- backward hops: blocks of the neighbours x - mu, transposed in registers
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int s = __ldg(nb + x * 8 + 4 + mu);
#pragma unroll
    for (int kt = 0; kt < NT; ++kt) {
      const uint4* base = frag + ((((size_t)s * 5 + 1 + mu) * NT + kt) * NT + rt) * TILE;
      const uint4 are = frag_transpose(__ldg(base + lane));
      const uint4 aim = frag_transpose(__ldg(base + 32 + lane));
      const uint32_t nl = adj ? 0u : s3mask(16 * kt), nh = adj ? 0u : s3mask(16 * kt + 8);
#pragma unroll
      for (int tl = 0; tl < T; ++tl) {
        uint32_t b0, b1;
        mrhs_bfrag<N>(c, s, kt, tl, nl, nh, b0, b1);
        mma_bf16(Q1[tl], are, b0, b1);
        mma_bf16(Q2[tl], aim, b0, b1);
      }
    }
  }
  // ---- epilogue: lane (g, t) owns rows r0 = 16rt + g, r1 = r0 + 8 of column 4tl + t
  const int r0 = 16 * rt + g, r1 = r0 + 8;
  const float s0 = (16 * rt < NV) ? 1.f : -1.f, s1 = (16 * rt + 8 < NV) ? 1.f : -1.f;
#pragma unroll
  for (int tl = 0; tl < T; ++tl) {
    const int q = kMrhsTile * tl + t;
    if (q >= c.R) continue;
    float2 y0 = make_float2(P1[tl][0] - P2[tl][1] + s0 * (Q1[tl][0] + Q2[tl][1]),
                            P1[tl][1] + P2[tl][0] + s0 * (Q1[tl][1] - Q2[tl][0]));
    float2 y1 = make_float2(P1[tl][2] - P2[tl][3] + s1 * (Q1[tl][2] + Q2[tl][3]),
                            P1[tl][3] + P2[tl][2] + s1 * (Q1[tl][3] - Q2[tl][2]));
    if (mu != 0.f) {
      const float2* xs = c.x + q * c.ldx + (size_t)x * N;
      const float2 v0 = __ldg(xs + r0), v1 = __ldg(xs + r1);
      const float m0 = adj ? mu : mu * s0, m1 = adj ? mu : mu * s1;
      y0.x -= m0 * v0.y; y0.y += m0 * v0.x;
      y1.x -= m1 * v1.y; y1.y += m1 * v1.x;
    }
    if (adj) {
      y0.x *= s0; y0.y *= s0;
      y1.x *= s1; y1.y *= s1;
    }
    float2* ys = c.y + q * c.ldy + (size_t)x * N;
    ys[r0] = y0;
    ys[r1] = y1;
  }
}

}  // namespace coarse
