// The shared-memory pipeline of the multi-RHS tensor-core apply, generic over where its sites
// come from and what happens to the results (a policy class):
//
//   struct Policy {
//     static constexpr bool kRuntimeT;                      // operators with fewer tiles than TACC
//     __device__ int ngroups(int P) const;                  // site groups of P sites
//     __device__ MrhsGroup group(int g, int P) const;       // blocks / vectors / sites of group g
//     __device__ int adjoint() const;
//     __device__ void finish(const MrhsGroup&, int x, int rt, const MrhsAcc<TACC>&) const;  // epilogue
//   };
//
// A CTA walks its site groups g = blockIdx.x + k * gridDim.x and for each the 9 items of Eq. (6):
// b = 0 self, 1..4 forward hop mu = b-1 (block of x, vector of x+mu), 5..8 backward hop mu = b-5
// (block of x-mu, vector of x-mu).  One producer warp brings each item's P blocks (fragment
// layout, one bulk copy each) and the P packed vector sets (one bulk copy each) into a ring of S
// shared-memory stages completing on the stage's "full" mbarrier; P * n/16 consumer warps (site
// p, 16-row tile rt) run the tensor-core products from shared memory and release the stage on
// its "empty" mbarrier.  All waits are bounded: on expiry the kernel raises *err, the producer
// drains its copies in flight, and all warps return.
#pragma once

#include "mrhs_core.cuh"
#include "pipe.cuh"

namespace coarse {

struct MrhsGroup {
  const uint4* frag;  // fragment-native blocks of the group's operator
  const int* nb;      // its neighbour table
  const uint2* xb;    // its packed vector fragments ([V][T][NT][32] uint2)
  int V;              // its sites
  int x0, np;         // first site of the group, sites in the group (<= P)
  int T;              // column tiles of the operator (<= the kernel's TACC)
  int tag;            // policy data (e.g. the operator index)
};

// Threads of a CTA (consumer warps + the producer warp) and the CTAs per SM to reserve registers
// for (at most 128 registers per thread).
__host__ __device__ constexpr int mrhs_threads(int N, int P) { return (P * (N / 16) + 1) * 32; }
__host__ __device__ constexpr int mrhs_min_blocks(int N, int P) {
  return 65536 / (mrhs_threads(N, P) * 128) > 0 ? 65536 / (mrhs_threads(N, P) * 128) : 1;
}

__host__ __device__ constexpr uint32_t mrhs_stage_bytes(int N, int P, int TACC) {
  return (uint32_t)P * (4u * N * N + (uint32_t)TACC * (N / 16) * 256u);
}

template <int N, int P, int TACC, class Policy>
__device__ __forceinline__ void mrhs_ring(const Policy& pol, int S, uint32_t SB, int* err) {
  constexpr int NT = N / 16, WC = P * NT;
  constexpr uint32_t BLK = 4u * N * N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
  uint64_t* empty = full + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = pol.ngroups(P);
  const int my_groups = (int)blockIdx.x < ngroups ? (ngroups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int items = my_groups * 9;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, WC);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == WC) {  // ---------------------------------------------------------- producer
    // lane p < P issues the block copy of site p of the group, lane P + p its vector copy; both
    // keep the site's neighbour row in registers for the group's 9 items.
    const int p = lane < P ? lane : lane - P;
    const bool active = lane < 2 * P;
    // the next group's description and neighbour rows are fetched one group ahead, so that
    // their latency never stalls the copies
    auto fetch = [&](int k, MrhsGroup& g, int4& lo, int4& hi) {
      const int gi = (int)blockIdx.x + k * (int)gridDim.x;
      if (gi >= ngroups) return;
      g = pol.group(gi, P);
      if (active && p < g.np) {
        const int x = g.x0 + p;
        lo = __ldg(reinterpret_cast<const int4*>(g.nb + x * 8));
        hi = __ldg(reinterpret_cast<const int4*>(g.nb + x * 8 + 4));
      }
    };
    MrhsGroup gr{}, gn{};
    int4 nb_lo = make_int4(0, 0, 0, 0), nb_hi = nb_lo, nx_lo = nb_lo, nx_hi = nb_lo;
    fetch(0, gn, nx_lo, nx_hi);
    int ok = 1;
    int it = 0;
    for (; it < items; ++it) {
      const int slot = it % S;
      const int b = it % 9;
      if (b == 0) {
        gr = gn;
        nb_lo = nx_lo;
        nb_hi = nx_hi;
        fetch(it / 9 + 1, gn, nx_lo, nx_hi);
      }
      if (it >= S && lane == 0) ok = mbar_wait_suspend(empty + slot, (uint32_t)((it / S - 1) & 1)) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      const uint32_t VB = (uint32_t)(Policy::kRuntimeT ? gr.T : TACC) * NT * 256u;
      unsigned char* st = smem + (size_t)slot * SB;
      if (lane == 0) mbar_expect_tx(full + slot, (uint32_t)gr.np * (BLK + VB));
      __syncwarp();
      if (active && p < gr.np) {
        const int x = gr.x0 + p;
        int src = x;  // source site of the vector: x (self), x + mu (forward), x - mu (backward)
        switch (b) {
          case 1: src = nb_lo.x; break;
          case 2: src = nb_lo.y; break;
          case 3: src = nb_lo.z; break;
          case 4: src = nb_lo.w; break;
          case 5: src = nb_hi.x; break;
          case 6: src = nb_hi.y; break;
          case 7: src = nb_hi.z; break;
          case 8: src = nb_hi.w; break;
        }
        if (lane < P) {
          const size_t blkid = b < 5 ? (size_t)x * 5 + b : (size_t)src * 5 + 1 + (b - 5);
          bulk_g2s(st + p * BLK, gr.frag + blkid * (BLK / 16), BLK, full + slot);
        } else {
          bulk_g2s(st + P * BLK + p * VB, gr.xb + (size_t)src * (VB / 8), VB, full + slot);
        }
      }
    }
    if (!ok && lane == 0) {
      atomicExch(err, 1);
      // drain the bulk copies this CTA still has in flight (bounded) before it exits
      for (int j = it - S < 0 ? 0 : it - S; j < it; ++j) mbar_wait(full + (j % S), (uint32_t)((j / S) & 1));
    }
    return;
  }

  // ---------------------------------------------------------------------------------- consumers
  const int p = warp / NT, rt = warp % NT;
  const int adj = pol.adjoint();
  MrhsAcc<TACC> acc;
  acc.zero();
  MrhsGroup gr{};
  int ok = 1;
  for (int it = 0; it < items; ++it) {
    const int slot = it % S;
    const int b = it % 9;
    if (b == 0) gr = pol.group((int)blockIdx.x + (it / 9) * (int)gridDim.x, P);
    if (!mbar_wait_suspend(full + slot, (uint32_t)((it / S) & 1))) ok = 0;
    if (!__all_sync(0xffffffffu, ok)) break;
    const bool valid = p < gr.np;
    const int Tn = Policy::kRuntimeT ? gr.T : TACC;  // compile-time for single-shape policies
    const uint32_t VB = (uint32_t)Tn * NT * 256u;
    const unsigned char* st = smem + (size_t)slot * SB;
    if (valid) {
      const uint4* blk = reinterpret_cast<const uint4*>(st + p * BLK);
      const uint2* vec = reinterpret_cast<const uint2*>(st + P * BLK + p * VB);
      if constexpr (Policy::kRuntimeT) {  // warp-uniform dispatch on the operator's tile count
        if (Tn == 1) mrhs_block<N, 1, TACC>(blk, vec, rt, b >= 5, adj, acc);
        else if (TACC >= 2 && Tn == 2) mrhs_block<N, (TACC >= 2 ? 2 : 1), TACC>(blk, vec, rt, b >= 5, adj, acc);
        else mrhs_block<N, TACC, TACC>(blk, vec, rt, b >= 5, adj, acc);
      } else {
        mrhs_block<N, TACC, TACC>(blk, vec, rt, b >= 5, adj, acc);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + slot);
    if (b == 8) {
      if (valid) pol.finish(gr, gr.x0 + p, rt, acc);
      acc.zero();
    }
  }
  if (!ok && lane == 0) atomicExch(err, 1);
}

}  // namespace coarse
