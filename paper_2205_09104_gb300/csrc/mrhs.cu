// Multi-right-hand-side apply Y = D_c X with BF16 blocks.
#include "common.cuh"

namespace coarse {

int launch_apply_mrhs_bf16(const coarse_op* op, const void* x, void* y, int nrhs, int adjoint, cudaStream_t s) {
  const size_t col = sizeof(float2) * (size_t)op->V * op->n;
  for (int c = 0; c < nrhs; ++c) {
    ApplyArgs a = make_apply_args(op, COARSE_PREC_BF16, (const char*)x + c * col, (char*)y + c * col);
    a.mu = adjoint ? -op->mu : op->mu;
    a.adjoint = adjoint;
    int rc = launch_apply(COARSE_PREC_BF16, op->n, a, s);
    if (rc != COARSE_OK) return rc;
  }
  return COARSE_OK;
}

}  // namespace coarse
