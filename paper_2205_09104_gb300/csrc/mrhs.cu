// Multi-right-hand-side apply Y = D_c X on tensor cores (BF16 blocks and vector fragments,
// FP32 accumulation), and the repacking of the BF16 blocks into the fragment-native layout
// it reads.  The per-site computation is in mrhs_core.cuh.
#include "mrhs_core.cuh"

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

constexpr int kMrhsWarps = 8;

template <int N, int T>
__global__ void __launch_bounds__(kMrhsWarps * 32, 2)
    k_apply_mrhs(const uint4* __restrict__ frag, const int* __restrict__ nb, MrhsCols c, int V, float mu, int adj) {
  constexpr int NT = N / 16;
  const int items = V * NT;
  for (int it = blockIdx.x * kMrhsWarps + (threadIdx.x >> 5); it < items; it += gridDim.x * kMrhsWarps)
    mrhs_rows<N, T>(frag, nb, c, it / NT, it % NT, mu, adj);
}

template <int N>
int launch_mrhs_n(const uint4* frag, const int* nb, const MrhsCols& c, int V, float mu, int adj, cudaStream_t s) {
  const int items = V * (N / 16);
  int grid = (items + kMrhsWarps - 1) / kMrhsWarps;
  const int cap = 2 * sm_count();
  if (grid > cap) grid = cap;
  const int T = (c.R + kMrhsTile - 1) / kMrhsTile;
  switch (T) {
    case 1: k_apply_mrhs<N, 1><<<grid, kMrhsWarps * 32, 0, s>>>(frag, nb, c, V, mu, adj); break;
    case 2: k_apply_mrhs<N, 2><<<grid, kMrhsWarps * 32, 0, s>>>(frag, nb, c, V, mu, adj); break;
    case 3: k_apply_mrhs<N, 3><<<grid, kMrhsWarps * 32, 0, s>>>(frag, nb, c, V, mu, adj); break;
    default: set_error("multi-RHS apply: %d columns in one pass", c.R); return COARSE_ERR_INVALID_ARG;
  }
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
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
  const long long col = (long long)op->V * op->n;
  const float mu = (float)(adjoint ? -op->mu : op->mu);
  constexpr int kPass = kMrhsTile * kMrhsMaxT;
  for (int c0 = 0; c0 < nrhs; c0 += kPass) {
    MrhsCols c;
    c.x = (const float2*)x + c0 * col;
    c.y = (float2*)y + c0 * col;
    c.ldx = c.ldy = col;
    c.R = nrhs - c0 < kPass ? nrhs - c0 : kPass;
    int rc;
    switch (op->n) {
      case 16: rc = launch_mrhs_n<16>((const uint4*)op->mrhs.ptr, op->nb, c, op->V, mu, adjoint, s); break;
      case 32: rc = launch_mrhs_n<32>((const uint4*)op->mrhs.ptr, op->nb, c, op->V, mu, adjoint, s); break;
      case 48: rc = launch_mrhs_n<48>((const uint4*)op->mrhs.ptr, op->nb, c, op->V, mu, adjoint, s); break;
      default: set_error("multi-RHS apply: unsupported n = %d", op->n); return COARSE_ERR_INVALID_ARG;
    }
    if (rc != COARSE_OK) return rc;
  }
  return COARSE_OK;
}

}  // namespace coarse
