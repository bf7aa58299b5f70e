// Block ingest (canonical FP64 Galerkin blocks -> internal 5-block storage in
// FP64 / FP32 / BF16), the sigma3 relation check and the block gradients.
#include "common.cuh"

namespace coarse {
namespace {

// out[x][b][i][j], b = 0 self, 1..4 forward hops.  One thread per complex entry.
__global__ void k_ingest(const double2* self_b, const double2* hop_b, int nhop, int V, int n, double2* o64,
                         float2* o32, cbf16* o16) {
  const size_t nn = (size_t)n * n;
  const size_t total = (size_t)V * 5 * nn;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t x = e / (5 * nn);
    const size_t r = e % (5 * nn);
    const int b = (int)(r / nn);
    const size_t ij = r % nn;
    const double2 v = (b == 0) ? self_b[x * nn + ij] : hop_b[(x * nhop + (b - 1)) * nn + ij];
    if (o64) o64[e] = v;
    if (o32) o32[e] = make_float2((float)v.x, (float)v.y);
    if (o16) {
      cbf16 c;
      c.x = __float2bfloat16_rn((float)v.x);
      c.y = __float2bfloat16_rn((float)v.y);
      o16[e] = c;
    }
  }
}

__device__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// out2[0] = max |defect|, out2[1] = max |entry|.  Defects: backward hop vs sigma3 F^H sigma3 of the
// forward hop of x - mu, and self block vs sigma3 A^H sigma3.
__global__ void k_gamma5_defect(const double2* self_b, const double2* hop_b, int V, int n, const int* nb,
                                double* out2) {
  const int nv = n / 2;
  const size_t nn = (size_t)n * n;
  const size_t total = (size_t)V * 5 * nn;
  double dmax = 0.0, emax = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t x = e / (5 * nn);
    const size_t r = e % (5 * nn);
    const int b = (int)(r / nn);
    const int i = (int)((r % nn) / n), j = (int)(r % n);
    const double s = ((i < nv) == (j < nv)) ? 1.0 : -1.0;
    double2 got, ref;
    if (b == 0) {
      got = self_b[x * nn + (size_t)i * n + j];
      const double2 t = self_b[x * nn + (size_t)j * n + i];
      ref = make_double2(s * t.x, -s * t.y);
    } else {
      const int mu = b - 1;
      got = hop_b[(x * 8 + 4 + mu) * nn + (size_t)i * n + j];
      const int xm = nb[x * 8 + 4 + mu];
      const double2 t = hop_b[((size_t)xm * 8 + mu) * nn + (size_t)j * n + i];
      ref = make_double2(s * t.x, -s * t.y);
      const double2 f = hop_b[(x * 8 + mu) * nn + (size_t)i * n + j];
      emax = fmax(emax, fmax(fabs(f.x), fabs(f.y)));
    }
    dmax = fmax(dmax, fmax(fabs(got.x - ref.x), fabs(got.y - ref.y)));
    emax = fmax(emax, fmax(fabs(got.x), fabs(got.y)));
    if (!isfinite(got.x) || !isfinite(got.y)) dmax = INFINITY;
  }
  for (int off = 16; off > 0; off >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(out2, dmax);
    atomic_max_nonneg(out2 + 1, emax);
  }
}

// G_self[x][i][j] = -lambda_x[i] conj(x_x[j]);  G_hop[x][d][i][j] = -lambda_x[i] conj(x_{nb(x,d)}[j]).
// nhop = 4 (gamma5-compressed input, backward hops derived as sigma3 F_{x-mu,mu}^H sigma3): the
// backward hop of y + mu depends on F_{y,mu} antilinearly, so its gradient folds onto the forward
// block as sigma3 G^H sigma3:  G4[y][mu][i][j] = -lambda_y[i] conj(x_{y+mu}[j])
//                                                 - s_i s_j x_y[i] conj(lambda_{y+mu}[j]).
// One thread per output entry; writes are coalesced along j.
__global__ void k_block_grad(const double2* lam, const double2* xv, const int* nb, int V, int n, int nhop,
                             double2* g_self, double2* g_hop) {
  const size_t nn = (size_t)n * n;
  const size_t nb_out = 1 + (size_t)nhop;
  const size_t total = (size_t)V * nb_out * nn;
  const int half = n / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t x = e / (nb_out * nn);
    const size_t r = e % (nb_out * nn);
    const int b = (int)(r / nn);
    const int i = (int)((r % nn) / n), j = (int)(r % n);
    const size_t src = (b == 0) ? x : (size_t)nb[x * 8 + (b - 1)];
    const double2 l = lam[x * n + i];
    const double2 v = xv[src * n + j];
    double2 g = make_double2(-(l.x * v.x + l.y * v.y), -(l.y * v.x - l.x * v.y));
    if (b > 0 && nhop == 4) {
      // - s_i s_j x_y[i] conj(lambda_{y+mu}[j]), y = x, y + mu = src
      const double2 xi = xv[x * n + i];
      const double2 lj = lam[src * n + j];
      const double sgn = ((i < half) == (j < half)) ? -1.0 : 1.0;
      g.x += sgn * (xi.x * lj.x + xi.y * lj.y);
      g.y += sgn * (xi.y * lj.x - xi.x * lj.y);
    }
    if (b == 0) g_self[x * nn + (size_t)i * n + j] = g;
    else g_hop[(x * nhop + (b - 1)) * nn + (size_t)i * n + j] = g;
  }
}

int grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

int launch_ingest(const double2* self_b, const double2* hop_b, int gamma5_only, int V, int n, const int* nb,
                  void* out64, void* out32, void* out16, cudaStream_t s) {
  (void)nb;
  const size_t total = (size_t)V * 5 * n * n;
  k_ingest<<<grid_for(total), 256, 0, s>>>(self_b, hop_b, gamma5_only ? 4 : 8, V, n, (double2*)out64,
                                           (float2*)out32, (cbf16*)out16);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_gamma5_defect(const double2* self_b, const double2* hop_b, int V, int n, const int* nb, double* out2,
                         cudaStream_t s) {
  COARSE_CUDA(cudaMemsetAsync(out2, 0, 2 * sizeof(double), s));
  const size_t total = (size_t)V * 5 * n * n;
  k_gamma5_defect<<<grid_for(total), 256, 0, s>>>(self_b, hop_b, V, n, nb, out2);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_block_grad(const double2* lam, const double2* x, const int* nb, int V, int n, int nhop, double2* g_self,
                      double2* g_hop, cudaStream_t s) {
  const size_t total = (size_t)V * (1 + nhop) * n * n;
  k_block_grad<<<grid_for(total), 256, 0, s>>>(lam, x, nb, V, n, nhop, g_self, g_hop);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace coarse
