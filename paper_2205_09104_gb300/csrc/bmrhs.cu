// Batched multi-right-hand-side stencil phases: the columns (solves) of each operator go through
// the tensor-core pipeline of mrhs_ring.cuh together, all operators of one n in one launch.
// The epilogue applies each column's own gate and polynomial-chain step (Sec. 3.3's q(A)v chain,
// as in the single-RHS stencil's epilogue).
#include "batch.cuh"
#include "mrhs_ring.cuh"

namespace coarse {
namespace {

template <int N>
struct BMrhsPolicy {
  static constexpr bool kRuntimeT = true;
  const BMApply* pa;  // the kernel's __grid_constant__ parameter
  int step;           // Arnoldi step of the phase (device counter, read once)
  __device__ int ngroups(int) const { return pa->total_groups; }
  __device__ MrhsGroup group(int g, int P) const {
    const BMApply& a = *pa;
    const int k = __ldg(a.grp_op + g);
    const BMOp& op = a.ops[a.idx[k]];
    MrhsGroup r;
    r.frag = static_cast<const uint4*>(op.frag);
    r.nb = op.nb;
    r.xb = static_cast<const uint2*>(op.xb);
    r.V = op.V;
    r.x0 = (g - a.grp_off[k]) * P;
    r.np = op.V - r.x0 < P ? op.V - r.x0 : P;
    r.T = op.T;
    r.tag = a.idx[k];
    return r;
  }
  __device__ int adjoint() const { return 0; }
  __device__ void finish(const MrhsGroup& gr, int x, int rt, const MrhsAcc<kMrhsMaxT>& acc) const {
    const BMApply& a = *pa;
    const BMOp& op = a.ops[gr.tag];
    const int lane = threadIdx.x & 31, t = lane & 3, g = lane >> 2;
    const int r0 = 16 * rt + g;
#pragma unroll
    for (int tl = 0; tl < kMrhsMaxT; ++tl) {
      if (tl >= gr.T) break;
      const int q = kMrhsTile * tl + t;
      if (q >= op.R) continue;
      const BSolve& s = a.S[op.s0 + q];
      if (!bgate(s, a.gate)) continue;
      const float2* xv = static_cast<const float2*>(bsel(s, a.xsel, step)) + (size_t)x * N;
      float2* yv = static_cast<float2*>(bsel(s, a.ysel, step)) + (size_t)x * N;
      float2 y[2];
      mrhs_rows_out<N, kMrhsMaxT>(acc, tl, rt, xv, op.mu, 0, y[0], y[1]);
      if (a.mode == APPLY_PLAIN) {
        yv[r0] = y[0];
        yv[r0 + 8] = y[1];
        continue;
      }
      // chain step: s' = s - c0 D s ; acc = acc + c1 s'  (first step: acc = c2 s + c1 s')
      const double2* cf = s.polyc + a.coef_off;
      const float2 c0 = make_float2((float)cf[0].x, (float)cf[0].y), c1 = make_float2((float)cf[1].x, (float)cf[1].y);
      float2* av = static_cast<float2*>(s.acc) + (size_t)x * N;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + 8 * h;
        const float2 xs = xv[r];
        const float2 sp = make_float2(xs.x - (c0.x * y[h].x - c0.y * y[h].y), xs.y - (c0.x * y[h].y + c0.y * y[h].x));
        float2 ac;
        if (a.mode == APPLY_POLY_FIRST) {
          const float2 c2 = make_float2((float)cf[2].x, (float)cf[2].y);
          ac = make_float2(c2.x * xs.x - c2.y * xs.y, c2.x * xs.y + c2.y * xs.x);
        } else {
          ac = av[r];
        }
        ac.x += c1.x * sp.x - c1.y * sp.y;
        ac.y += c1.x * sp.y + c1.y * sp.x;
        yv[r] = sp;
        av[r] = ac;
      }
    }
  }
};

template <int N, int P>
__global__ void __launch_bounds__(mrhs_threads(N, P), mrhs_min_blocks(N, P)) kb_apply_mrhs(const __grid_constant__ BMApply a, int S, uint32_t SB) {
  const BMrhsPolicy<N> pol{&a, *a.step};
  mrhs_ring<N, P, kMrhsMaxT>(pol, S, SB, a.err);
}

// input columns of every operator -> packed BF16 B fragments (zeros for gated-off columns and
// for the columns R .. 4T-1 of the last tile); layout as k_pack_mrhs_x
__global__ void kb_pack_mrhs_x(BMApply a, int nops, const int* __restrict__ word_off, int total) {
  const int step = *a.step;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int k = find_solve(word_off, nops, i);
    const BMOp& op = a.ops[k];
    const int NT = op.n / 16;
    const int local = i - word_off[k];
    const int w = local & 1, lane = (local >> 1) & 31;
    int rest = local >> 6;
    const int kt = rest % NT;
    rest /= NT;
    const int tl = rest % op.T;
    const int site = rest / op.T;
    const int g = lane >> 2, t = lane & 3;
    const int q = kMrhsTile * tl + (g >> 1);
    uint32_t v = 0u;
    if (q < op.R) {
      const BSolve& s = a.S[op.s0 + q];
      if (bgate(s, a.gate)) {
        const float2* x = static_cast<const float2*>(bsel(s, a.xsel, step)) + (size_t)site * op.n;
        const float4 e = *reinterpret_cast<const float4*>(x + 16 * kt + 2 * t + 8 * w);
        v = (g & 1) ? bf2_bits(e.y, e.w) : bf2_bits(e.x, e.z);
      }
    }
    static_cast<uint32_t*>(op.xb)[local] = v;
  }
}

constexpr int kBMaxSmem = 200 * 1024;

template <int N, int P>
int launch_bm(int S, const BMApply& a, cudaStream_t s) {
  constexpr int THREADS = (P * (N / 16) + 1) * 32;
  static bool attr = false;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(kb_apply_mrhs<N, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBMaxSmem));
    attr = true;
  }
  const uint32_t SB = mrhs_stage_bytes(N, P, kMrhsMaxT);
  S = S < 2 ? 2 : (S > 8 ? 8 : S);
  while (S > 2 && (size_t)S * SB + 16 * S > (size_t)kBMaxSmem) --S;
  const size_t smem = (size_t)S * SB + 2 * S * sizeof(uint64_t);
  int per_sm = 0;
  COARSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_apply_mrhs<N, P>, THREADS, smem));
  if (per_sm < 1) {
    set_error("batched multi-RHS apply: no CTA fits (%zu bytes of shared memory)", smem);
    return COARSE_ERR_INVALID_ARG;
  }
  int grid = per_sm * sm_count();
  if (grid > a.total_groups) grid = a.total_groups;
  if (grid < 1) return COARSE_OK;
  kb_apply_mrhs<N, P><<<grid, THREADS, smem, s>>>(a, S, SB);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace

int launch_bpack_mrhs(const BMApply& a, int nops, const int* word_off, int total_words, cudaStream_t s) {
  if (total_words <= 0) return COARSE_OK;
  int grid = (total_words + 255) / 256;
  if (grid > sm_count() * 16) grid = sm_count() * 16;
  kb_pack_mrhs_x<<<grid, 256, 0, s>>>(a, nops, word_off, total_words);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_bapply_mrhs(int n, int P, int S, const BMApply& a, cudaStream_t s) {
  switch (n * 16 + P) {
    case 16 * 16 + 2: return launch_bm<16, 2>(S, a, s);
    case 16 * 16 + 4: return launch_bm<16, 4>(S, a, s);
    case 32 * 16 + 1: return launch_bm<32, 1>(S, a, s);
    case 32 * 16 + 2: return launch_bm<32, 2>(S, a, s);
    case 48 * 16 + 1: return launch_bm<48, 1>(S, a, s);
    case 48 * 16 + 2: return launch_bm<48, 2>(S, a, s);
  }
  set_error("batched multi-RHS apply: no kernel for n = %d with %d sites per stage", n, P);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace coarse
