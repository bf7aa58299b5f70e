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
// load per lane per tile and plane, conflict-free from shared memory.  The transpose F^T of a
// tile is made in registers with movmatrix (a0' = T(a0), a1' = T(a2), a2' = T(a1), a3' = T(a3)).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace coarse {

constexpr int kMrhsTile = 4;    // columns per tensor-core tile (B operand is 8 wide: re, im of 4 columns)
constexpr int kMrhsMaxT = 3;    // tiles per pass: up to 12 columns
constexpr int kMrhsPass = kMrhsTile * kMrhsMaxT;
constexpr int kMrhsColumns = kMrhsPass;  // columns one pass (and one batched operator) can carry
constexpr int kTcPass = 16;              // columns of one pass of the tcgen05 kernel (4 tiles)

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

// Accumulators of one warp: output rows 16rt .. 16rt+15, T column tiles.
template <int T>
struct MrhsAcc {
  float P1[T][4], P2[T][4], Q1[T][4], Q2[T][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int tl = 0; tl < T; ++tl)
#pragma unroll
      for (int i = 0; i < 4; ++i) P1[tl][i] = P2[tl][i] = Q1[tl][i] = Q2[tl][i] = 0.f;
  }
};

// Fragment-native BF16 vectors (built by k_pack_mrhs_x from the complex64 columns): for each
// site, column tile tl and k tile kt, lane (g, t) holds the two B-fragment registers
//   b0 = part (g & 1 ? Im : Re) of x_{4tl + g/2}[16kt + 2t + {0, 1}],   b1 = the same at + 8,
// as one uint2 at index (tl * NT + kt) * 32 + lane; columns >= R hold zeros.  One site of T tiles
// is T * NT * 256 bytes, contiguous.
__device__ __forceinline__ uint32_t s3mask(int k0, int nv) { return k0 < nv ? 0u : 0x80008000u; }

// One staged block (all NT x NT tiles, fragment layout) times the staged vectors of its source site.
// Forward / self blocks (bwd = 0): P += F w with w = (adj ? s3 x : x), rows of tile rt.
// Backward blocks (bwd = 1): Q += F^T-products on (adj ? x : s3 x), columns of tile rt (F^H w).
// Column tiles 0 .. T-1 of accumulators sized TA >= T (T is a compile-time count so that the
// unrolled loops carry no branches).
template <int N, int T, int TA = T>
__device__ __forceinline__ void mrhs_block(const uint4* blk, const uint2* vec, int rt, int bwd, int adj,
                                           MrhsAcc<TA>& acc) {
  constexpr int NT = N / 16;
  const int lane = threadIdx.x & 31;
  const int flip = bwd ? !adj : adj;  // sigma3 on the B operand
#pragma unroll
  for (int kt = 0; kt < NT; ++kt) {
    uint4 are, aim;
    if (!bwd) {
      are = blk[((rt * NT + kt) * 2 + 0) * 32 + lane];
      aim = blk[((rt * NT + kt) * 2 + 1) * 32 + lane];
    } else {
      are = frag_transpose(blk[((kt * NT + rt) * 2 + 0) * 32 + lane]);
      aim = frag_transpose(blk[((kt * NT + rt) * 2 + 1) * 32 + lane]);
    }
    const uint32_t nl = flip ? s3mask(16 * kt, N / 2) : 0u, nh = flip ? s3mask(16 * kt + 8, N / 2) : 0u;
#pragma unroll
    for (int tl = 0; tl < T; ++tl) {
      const uint2 bv = vec[(tl * NT + kt) * 32 + lane];
      const uint32_t b0 = bv.x ^ nl, b1 = bv.y ^ nh;
      if (!bwd) {
        mma_bf16(acc.P1[tl], are, b0, b1);
        mma_bf16(acc.P2[tl], aim, b0, b1);
      } else {
        mma_bf16(acc.Q1[tl], are, b0, b1);
        mma_bf16(acc.Q2[tl], aim, b0, b1);
      }
    }
  }
}

// Output rows r0 = 16rt + g and r1 = r0 + 8 of column q = 4tl + t:
//   y = o (P + s3 Q + i mu' v),  v = (adj ? x : s3 x),  o = (adj ? s3 : 1),
// with mu' already signed (-mu for the adjoint).  Returns the two complex values.
template <int N, int T>
__device__ __forceinline__ void mrhs_rows_out(const MrhsAcc<T>& acc, int tl, int rt, const float2* xsite, float mu,
                                              int adj, float2& y0, float2& y1) {
  constexpr int NV = N / 2;
  const int g = (threadIdx.x & 31) >> 2;
  const float s0 = (16 * rt < NV) ? 1.f : -1.f, s1 = (16 * rt + 8 < NV) ? 1.f : -1.f;
  y0 = make_float2(acc.P1[tl][0] - acc.P2[tl][1] + s0 * (acc.Q1[tl][0] + acc.Q2[tl][1]),
                   acc.P1[tl][1] + acc.P2[tl][0] + s0 * (acc.Q1[tl][1] - acc.Q2[tl][0]));
  y1 = make_float2(acc.P1[tl][2] - acc.P2[tl][3] + s1 * (acc.Q1[tl][2] + acc.Q2[tl][3]),
                   acc.P1[tl][3] + acc.P2[tl][2] + s1 * (acc.Q1[tl][3] - acc.Q2[tl][2]));
  if (mu != 0.f) {
    const int r0 = 16 * rt + g;
    const float2 v0 = __ldg(xsite + r0), v1 = __ldg(xsite + r0 + 8);
    const float m0 = adj ? mu : mu * s0, m1 = adj ? mu : mu * s1;
    y0.x -= m0 * v0.y; y0.y += m0 * v0.x;
    y1.x -= m1 * v1.y; y1.y += m1 * v1.x;
  }
  if (adj) {
    y0.x *= s0; y0.y *= s0;
    y1.x *= s1; y1.y *= s1;
  }
}

}  // namespace coarse
