// coarse_solve_batched: independent solves of uneven operators.
#include "common.cuh"
#include "solver.cuh"

extern "C" int coarse_solve_batched(coarse_op* const* ops, int nops, const void* const* b, void* const* x,
                                    const int* nrhs, const coarse_solve_params* params, coarse_solve_info* infos,
                                    void* stream) {
  if (nops < 0 || (nops > 0 && (!ops || !b || !x || !nrhs || !params))) {
    coarse::set_error("coarse_solve_batched: NULL array or negative nops");
    return COARSE_ERR_INVALID_ARG;
  }
  int worst = COARSE_OK;
  size_t at = 0;
  for (int i = 0; i < nops; ++i) {
    int rc = coarse_solve(ops[i], b[i], x[i], nrhs[i], params, infos ? infos + at : nullptr, stream);
    at += nrhs[i] > 0 ? nrhs[i] : 0;
    if (rc != COARSE_OK && rc != COARSE_ERR_NOT_CONVERGED) return rc;
    if (rc != COARSE_OK) worst = rc;
  }
  return worst;
}
