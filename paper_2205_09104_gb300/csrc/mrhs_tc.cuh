// The tcgen05 multi-right-hand-side apply (mrhs_tc.cu): arguments and launchers.
#pragma once

#include <cstdint>

#include "mrhs_core.cuh"

namespace coarse {

struct TcArgs {
  const unsigned char* blk;  // BF16 blocks as core-matrix planes, [V * 5][2][n * n] (k_pack_tc)
  const int* nb;             // [V][8]
  const float2* x;           // column q at x + q * ldx (complex64 [V][n])
  unsigned char* xv;         // packed columns, [V][2][8T][n] BF16 (written by the launcher's pack)
  float2* y;
  long long ldx, ldy;
  int R;                     // columns of this pass (1 .. 4T, T <= 4)
  int V, n;
  int S;                     // pipeline stages (set by the launcher)
  float mu;                  // signed twisted mass (-mu for the adjoint)
  int adj;
  int* err;
};

// Refresh the core-matrix planes from the BF16 blocks ([nblocks][n][n] complex BF16).
int launch_pack_tc(const void* bf16_blocks, void* dst, long long nblocks, int n, cudaStream_t s);
// Pack the R columns of a.x and apply (n = 32 or 48, T = 1 .. 4 column tiles of 4), with
// ctas_per_sm = 1 .. 3 CTAs per SM (3 only for T <= 2) and S stages (S <= 0: as many as fit).
int launch_apply_mrhs_tc(TcArgs a, int T, int ctas_per_sm, int S, cudaStream_t s);

}  // namespace coarse
