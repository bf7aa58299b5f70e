// Multi-right-hand-side apply Y = D_c X on the fifth-generation tensor cores (tcgen05.mma: BF16
// operands read from shared memory by the tensor core, FP32 accumulators in tensor memory) for
// n = 32 and 48, with the packing of the blocks and of the columns into its operand layout.
//
// Per site x the product is Eq. (6)'s nine block-vector products: the self block, the forward
// blocks F_{x,mu} applied to x_{x+mu} and the backward blocks sigma3 F_{x-mu,mu}^H sigma3 (only
// the forward hops are stored, Sec. 4.2) applied to x_{x-mu}.
//
// Complex as real, one MMA per plane.  With F = Fr + i Fi and the B operand [Xr | Xi] (the real
// parts of the 4T padded columns, then their imaginary parts: MMA width N = 8T)
//   Fr [Xr|Xi] = [Fr Xr | Fr Xi],  Fi [Xr|Xi] = [Fi Xr | Fi Xi]  ->  F X = (Fr Xr - Fi Xi) + i (Fr Xi + Fi Xr),
// and for a backward hop F^H W = (Fr^T Wr + Fi^T Wi) + i (Fr^T Wi - Fi^T Wr): the same planes read
// transposed.  The sigma3 of a hop acts on the B operand (a second, sign-flipped copy of every
// column set) and on the output rows (epilogue).  tcgen05.mma needs M >= 64, so each plane is
// one M = 64 operand; for n = 48 its rows 48..63 are whatever shared memory follows the plane
// (in bounds: the ring is followed by a pad), and those accumulator rows are never read.
//
// Block layout (global and shared, one bulk copy per block), 8 x 8 BF16 core matrices:
//   byte ((p * G + ri) * G + ci) * 128 + 16 r + 2 c  holds plane p of F[8 ri + r][8 ci + c],  G = n / 8.
// Read K-major (forward: rows of F along M) the core matrices of a row group are adjacent along
// K and row groups are G * 128 bytes apart; read MN-major (backward: F^T, columns of F along M)
// the M groups are 128 bytes apart and the K groups G * 128.  In both forms the descriptor's
// leading byte offset is the stride of core matrices along K and its stride byte offset the one
// along M or N (checked on the device: an in-bounds product of known operands), so one copy of a
// block serves both products; the major bit of the instruction, the two offsets and the start
// of each 16-deep K step differ.
//
// Column layout (packed per call by k_pack_tc_x): per site two variants v (0: x, 1: sigma3 x),
// each the K-major B operand of N = 8T rows and K = n: byte ((v * T + ni) * G + ki) * 128 + 16 r
// + 2 c holds row 8 ni + r (column j < 4T: Re x_j, else Im x_{j - 4T}; zero for padded columns)
// at entry 8 ki + c.
//
// Accumulators of an M = 64 product occupy tensor-memory lanes 0..15 of each 32-lane quarter
// (row 16 e + l in lane 32 e + l), also checked on the device.
//
// Pipeline (one CTA of 9 warps, persistent over sites x = blockIdx.x + k gridDim.x): warp 0
// lane 0 brings each of a site's 9 items (block + column variant, two bulk copies) into one of
// two rings of shared-memory stages ("full" mbarriers): self and forward hops into one,
// backward hops into the other, so that every stage's consumers take each of its phases in
// turn (a parity wait never sees a phase two ahead).  Warps 1..4 issue the MMAs, one lane each, and
// each owns one of a site's four accumulators (forward / backward hops x real / imaginary
// plane): a thread's tcgen05.mma stream advances by one instruction about every 160 cycles
// whatever M, N or the dependences between them (measured), so the MMAs of a site are spread
// over four issuing threads.  Each issuer releases a stage through tcgen05.commit ("empty",
// two arrivals: both planes of the item) and, after its last item of the site, commits the
// accumulator set to the epilogue ("acc full", four arrivals).  Warps 5..8 (one per
// tensor-memory lane quarter) read the set in chunks of four columns, combine and store the
// site's output rows, and free the set ("acc empty").  Every wait is bounded: on expiry the
// kernel raises *err, drains its bulk copies and MMAs (bounded again), frees its tensor memory
// and returns.
#include <cstdint>
#include <cstdio>

#include "mrhs_tc.cuh"
#include "pipe.cuh"

namespace coarse {
namespace {

constexpr int kTcThreads = 288;
constexpr uint32_t kTcPad = 2048;      // shared memory after the ring (over-read of M = 64 operands)

// Stages of the self / forward ring out of S in all (the rest hold backward hops), >= 2 each.
__host__ __device__ constexpr int tc_split(int S) {
  return (5 * S + 4) / 9 < 2 ? 2 : ((5 * S + 4) / 9 > S - 2 ? S - 2 : (5 * S + 4) / 9);
}

// Tensor-memory columns: 2 accumulator sets x 4 accumulators of width N = 8T, in slots of 16
// columns (T <= 2: 128 columns per CTA, up to 3 CTAs per SM) or 32 (T = 3, 4: 256, up to 2).
__host__ __device__ constexpr uint32_t tc_slot(int T) { return T <= 2 ? 16u : 32u; }
__host__ __device__ constexpr uint32_t tc_cols(int T) { return 8u * tc_slot(T); }

// shared-memory matrix descriptor, no swizzle: lbo = byte stride of core matrices along K, sbo =
// along M (A) or N (B)
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);  // version 1, no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, B K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// BF16 blocks [V][5][n][n] (complex, re in the low half) -> the core-matrix planes above.  One
// thread per block, row and entry pair.
__global__ void k_pack_tc(const uint32_t* __restrict__ src, uint16_t* __restrict__ dst, long long nblocks, int n) {
  const int G = n / 8, HP = n / 2;
  const long long total = nblocks * n * HP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int kp = (int)(i % HP);
    const long long rest = i / HP;
    const int a = (int)(rest % n);
    const long long blk = rest / n;
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(src + (blk * n + a) * n + 2 * kp));
    const int k = 2 * kp;
    const size_t off = (size_t)blk * 2 * n * n + (size_t)(((a >> 3) * G + (k >> 3)) * 64 + (a & 7) * 8 + (k & 7));
    // plane 0: real parts (low halves), plane 1: imaginary parts (high halves)
    *reinterpret_cast<uint32_t*>(dst + off) = __byte_perm(u.x, u.y, 0x5410);
    *reinterpret_cast<uint32_t*>(dst + off + (size_t)n * n) = __byte_perm(u.x, u.y, 0x7632);
  }
}

// complex64 columns x + q*ldx (q < R) -> the two B-operand variants of every site (layout
// above).  One thread per site, padded column q < 4T and entry pair kp.
__global__ void k_pack_tc_x(const float2* __restrict__ x, long long ldx, int R, int T, int V, int n,
                            uint16_t* __restrict__ xv) {
  const int G = n / 8, HP = n / 2, NV = n / 2, C = 4 * T;
  const long long total = (long long)V * C * HP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int kp = (int)(i % HP);
    const long long rest = i / HP;
    const int q = (int)(rest % C);
    const long long site = rest / C;
    uint32_t re = 0u, im = 0u;
    if (q < R) {
      const float4 e = __ldg(reinterpret_cast<const float4*>(x + q * ldx + site * n + 2 * kp));
      re = bf2_bits(e.x, e.z);
      im = bf2_bits(e.y, e.w);
    }
    const int k = 2 * kp;
    const uint32_t flip = k < NV ? 0u : 0x80008000u;  // sigma3: entries of the second half negated
    uint16_t* base = xv + (size_t)site * 2 * (8 * T) * n;
    const size_t vstride = (size_t)(8 * T) * n;
    const int jr = q, ji = C + q;
    const size_t o_r = (size_t)(((jr >> 3) * G + (k >> 3)) * 64 + (jr & 7) * 8 + (k & 7));
    const size_t o_i = (size_t)(((ji >> 3) * G + (k >> 3)) * 64 + (ji & 7) * 8 + (k & 7));
    *reinterpret_cast<uint32_t*>(base + o_r) = re;
    *reinterpret_cast<uint32_t*>(base + o_i) = im;
    *reinterpret_cast<uint32_t*>(base + vstride + o_r) = re ^ flip;
    *reinterpret_cast<uint32_t*>(base + vstride + o_i) = im ^ flip;
  }
}

template <int N, int T>
__global__ void __launch_bounds__(kTcThreads, 2) k_apply_mrhs_tc(const __grid_constant__ TcArgs a) {
  constexpr int G = N / 8, KS = N / 16, NN = 8 * T;
  constexpr uint32_t PLANE = (uint32_t)N * N * 2, BLK = 2 * PLANE, VB = (uint32_t)NN * N * 2, SB = BLK + VB;
  constexpr uint32_t SBO = (uint32_t)G * 128;
  constexpr uint32_t ID_K = tc_idesc(64, NN, 0), ID_MN = tc_idesc(64, NN, 1);
  constexpr uint32_t SLOT = tc_slot(T), COLS = tc_cols(T);
  extern __shared__ __align__(1024) unsigned char smem[];
  const int S = a.S, Sf = tc_split(S), Sb = S - Sf;  // stages [0, Sf): forward ring, [Sf, S): backward
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB + kTcPad);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;   // [2]
  uint64_t* acce = accf + 2;    // [2]
  uint64_t* done = acce + 2;    // [4]: each MMA issuer's final commit
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_sites = (int)blockIdx.x < a.V ? (a.V - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int items = my_sites * 9;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 2);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accf + i, 4);
      mbar_init(acce + i, 4);
    }
    for (int i = 0; i < 4; ++i) mbar_init(done + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {  // ------------------------------------------------------------ producer
    if (lane == 0) {
      int ok = 1, it = 0, jf = 0, jb = 0;  // items issued per ring
      // neighbour rows of the current and (prefetched) next site
      int4 lo = make_int4(0, 0, 0, 0), hi = lo, nlo = lo, nhi = lo;
      if (my_sites > 0) {
        nlo = __ldg(reinterpret_cast<const int4*>(a.nb + (size_t)blockIdx.x * 8));
        nhi = __ldg(reinterpret_cast<const int4*>(a.nb + (size_t)blockIdx.x * 8 + 4));
      }
      for (; it < items; ++it) {
        const int b = it % 9, sk = it / 9;
        const int x = (int)blockIdx.x + sk * (int)gridDim.x;
        const int bw = b >= 5, Sx = bw ? Sb : Sf, j = bw ? jb : jf;
        const int slot = (bw ? Sf : 0) + j % Sx;
        if (it % 9 == 0) {
          lo = nlo;
          hi = nhi;
          if (sk + 1 < my_sites) {
            const int xn = x + (int)gridDim.x;
            nlo = __ldg(reinterpret_cast<const int4*>(a.nb + (size_t)xn * 8));
            nhi = __ldg(reinterpret_cast<const int4*>(a.nb + (size_t)xn * 8 + 4));
          }
        }
        if (j >= Sx && !mbar_wait_suspend(empty + slot, (uint32_t)((j / Sx - 1) & 1))) {
          ok = 0;
          break;
        }
        if (bw) ++jb;
        else ++jf;
        int src = x;
        switch (b) {
          case 1: src = lo.x; break;
          case 2: src = lo.y; break;
          case 3: src = lo.z; break;
          case 4: src = lo.w; break;
          case 5: src = hi.x; break;
          case 6: src = hi.y; break;
          case 7: src = hi.z; break;
          case 8: src = hi.w; break;
        }
        const size_t blkid = b < 5 ? (size_t)x * 5 + b : (size_t)src * 5 + 1 + (b - 5);
        const int v = (b < 5) ? a.adj : !a.adj;  // sigma3 on the columns (forward: adjoint only)
        unsigned char* st = smem + (size_t)slot * SB;
        mbar_expect_tx(full + slot, SB);
        bulk_g2s(st, a.blk + blkid * BLK, BLK, full + slot);
        bulk_g2s(st + BLK, a.xv + ((size_t)src * 2 + v) * VB, VB, full + slot);
      }
      if (!ok) {
        atomicExch(a.err, 1);
        // drain the copies still in flight in either ring (bounded)
        for (int k = jf - Sf < 0 ? 0 : jf - Sf; k < jf; ++k) mbar_wait(full + k % Sf, (uint32_t)((k / Sf) & 1));
        for (int k = jb - Sb < 0 ? 0 : jb - Sb; k < jb; ++k) mbar_wait(full + Sf + k % Sb, (uint32_t)((k / Sb) & 1));
      }
    }
  } else if (warp <= 4) {  // --------------------------------------------------- MMA issuers
    if (lane == 0) {
      // issuer (bwd, p): items of one hop direction type (self + forward: 0..4, backward: 5..8),
      // plane p, into its own accumulator
      const int bwd = (warp - 1) >> 1, p = (warp - 1) & 1;
      const int b0 = bwd ? 5 : 0, b1 = bwd ? 9 : 5;
      int ok = 1;
      const uint32_t s0 = smem_u32(smem);
      for (int sk = 0; sk < my_sites && ok; ++sk) {
        const int buf = sk & 1;
        if (sk >= 2) {
          if (!mbar_wait_suspend(acce + buf, (uint32_t)((sk / 2 - 1) & 1))) { ok = 0; break; }
          tc_fence_after();
        }
        const uint32_t d = tmem + (uint32_t)buf * 4u * SLOT + (uint32_t)(bwd * 2 + p) * SLOT;
        const int Sx = bwd ? Sb : Sf, cnt = b1 - b0;
        for (int b = b0; b < b1; ++b) {
          const int j = sk * cnt + (b - b0), slot = (bwd ? Sf : 0) + j % Sx;
          if (!mbar_wait_suspend(full + slot, (uint32_t)((j / Sx) & 1))) { ok = 0; break; }
          tc_fence_after();
          const uint32_t st = s0 + (uint32_t)slot * SB;
#pragma unroll
          for (int s = 0; s < KS; ++s) {
            const uint64_t ad = bwd ? tc_sdesc(st + p * PLANE + 2u * s * SBO, SBO, 128u)    // F^T: K stride G*128
                                    : tc_sdesc(st + p * PLANE + 256u * s, 128u, SBO);       // F: K stride 128
            const uint64_t bd = tc_sdesc(st + BLK + 256u * s, 128u, SBO);
            tc_mma(d, ad, bd, bwd ? ID_MN : ID_K, (s > 0 || b != b0) ? 1u : 0u);
          }
          tc_commit(empty + slot);
        }
        if (ok) tc_commit(accf + buf);
      }
      if (!ok) atomicExch(a.err, 1);
      tc_commit(done + (warp - 1));  // completes when every MMA this thread issued has completed
      mbar_wait(done + (warp - 1), 0);
    }
  } else {  // ------------------------------------------------------------------- epilogue
    const int e = warp & 3;                   // tensor-memory lane quarter of this warp
    const int r = lane < 16 ? 16 * e + lane : -1;  // output row held by this thread's lane
    const float s = (r >= 0 && r < N / 2) ? 1.f : -1.f;
    const float m = a.adj ? a.mu : a.mu * s;
    int ok = 1;
    for (int sk = 0; sk < my_sites; ++sk) {
      const int buf = sk & 1;
      if (!mbar_wait_suspend(accf + buf, (uint32_t)((sk / 2) & 1))) ok = 0;
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)buf * 4u * SLOT;
      const int x = (int)blockIdx.x + sk * (int)gridDim.x;
      constexpr int C = 4 * T;
      // four columns at a time: for column q the real parts sit in accumulator column q, the
      // imaginary parts in column C + q, of each of the four accumulators
#pragma unroll
      for (int q0 = 0; q0 < C; q0 += 4) {
        float pr[2][4], pi[2][4], qr[2][4], qi[2][4];
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
          tc_ld4(base + (uint32_t)pl * SLOT + (uint32_t)q0, pr[pl]);
          tc_ld4(base + (uint32_t)pl * SLOT + (uint32_t)(C + q0), pi[pl]);
          tc_ld4(base + (uint32_t)(2 + pl) * SLOT + (uint32_t)q0, qr[pl]);
          tc_ld4(base + (uint32_t)(2 + pl) * SLOT + (uint32_t)(C + q0), qi[pl]);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (r >= 0 && r < N) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int q = q0 + j;
            if (q >= a.R) break;
            // forward F w and backward F^H w' of column q, then y = o (fwd + s bwd + i mu' v)
            float yr = pr[0][j] - pi[1][j] + s * (qr[0][j] + qi[1][j]);
            float yi = pi[0][j] + pr[1][j] + s * (qi[0][j] - qr[1][j]);
            if (a.mu != 0.f) {
              const float2 v = __ldg(a.x + q * a.ldx + (size_t)x * N + r);
              yr -= m * v.y;
              yi += m * v.x;
            }
            if (a.adj) {
              yr *= s;
              yi *= s;
            }
            a.y[q * a.ldy + (size_t)x * N + r] = make_float2(yr, yi);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + buf);
    }
    if (!ok && lane == 0) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  }
}

template <int N, int T>
int launch_tc_nt(TcArgs a, int ctas_per_sm, int S, cudaStream_t s) {
  constexpr uint32_t SB = 4u * N * N + 16u * T * N;
  // ctas_per_sm CTAs share the SM's shared memory; the shared memory of each is also at least
  // what keeps one more CTA (and one more tensor-memory allocation) off the SM
  // registers (9 warps of up to 72) allow 3 CTAs per SM; tensor memory 512 columns
  if (ctas_per_sm < 1 || ctas_per_sm > 3 || ctas_per_sm * tc_cols(T) > 512u) {
    set_error("tcgen05 multi-RHS apply: %d CTAs per SM with %u tensor-memory columns each", ctas_per_sm, tc_cols(T));
    return COARSE_ERR_INVALID_ARG;
  }
  const size_t sm_bytes = 228u * 1024u, reserve = 1024u;
  const size_t budget = sm_bytes / ctas_per_sm - reserve > 210u * 1024u ? 210u * 1024u : sm_bytes / ctas_per_sm - reserve;
  const size_t floor_bytes = sm_bytes / (ctas_per_sm + 1) + 1024u;
  const size_t fixed = kTcPad + (2 * 32 + 8) * sizeof(uint64_t) + 16;
  if (S <= 0) S = (int)((budget - fixed) / SB);
  S = S < 4 ? 4 : (S > 32 ? 32 : S);  // two rings of at least 2 stages
  while (S > 4 && S * SB + fixed > budget) --S;
  a.S = S;
  size_t smem = (size_t)S * SB + fixed;
  if (smem < floor_bytes) smem = floor_bytes;
  if (smem > budget) {
    set_error("tcgen05 multi-RHS apply: %zu bytes of shared memory for %d CTAs per SM", smem, ctas_per_sm);
    return COARSE_ERR_INVALID_ARG;
  }
  static bool attr = false;
  if (!attr) {
    COARSE_CUDA(cudaFuncSetAttribute(k_apply_mrhs_tc<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
    attr = true;
  }
  int grid = ctas_per_sm * sm_count();
  if (grid > a.V) grid = a.V;
  k_apply_mrhs_tc<N, T><<<grid, kTcThreads, smem, s>>>(a);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

}  // namespace

int launch_pack_tc(const void* bf16_blocks, void* dst, long long nblocks, int n, cudaStream_t s) {
  const long long total = nblocks * n * (n / 2);
  long long grid = (total + 255) / 256;
  if (grid > (long long)sm_count() * 16) grid = (long long)sm_count() * 16;
  k_pack_tc<<<(int)grid, 256, 0, s>>>((const uint32_t*)bf16_blocks, (uint16_t*)dst, nblocks, n);
  note_launch();
  COARSE_CUDA(cudaGetLastError());
  return COARSE_OK;
}

int launch_apply_mrhs_tc(TcArgs a, int T, int ctas_per_sm, int S, cudaStream_t s) {
  {
    const long long total = (long long)a.V * 4 * T * (a.n / 2);
    long long grid = (total + 255) / 256;
    if (grid > (long long)sm_count() * 16) grid = (long long)sm_count() * 16;
    k_pack_tc_x<<<(int)grid, 256, 0, s>>>(a.x, a.ldx, a.R, T, a.V, a.n, (uint16_t*)a.xv);
    note_launch();
    COARSE_CUDA(cudaGetLastError());
  }
  const int key = a.n * 8 + T;
  switch (key) {
    case 32 * 8 + 1: return launch_tc_nt<32, 1>(a, ctas_per_sm, S, s);
    case 32 * 8 + 2: return launch_tc_nt<32, 2>(a, ctas_per_sm, S, s);
    case 32 * 8 + 3: return launch_tc_nt<32, 3>(a, ctas_per_sm, S, s);
    case 48 * 8 + 1: return launch_tc_nt<48, 1>(a, ctas_per_sm, S, s);
    case 48 * 8 + 2: return launch_tc_nt<48, 2>(a, ctas_per_sm, S, s);
    case 48 * 8 + 3: return launch_tc_nt<48, 3>(a, ctas_per_sm, S, s);
    case 32 * 8 + 4: return launch_tc_nt<32, 4>(a, ctas_per_sm, S, s);
    case 48 * 8 + 4: return launch_tc_nt<48, 4>(a, ctas_per_sm, S, s);
  }
  set_error("tcgen05 multi-RHS apply: unsupported n = %d with %d column tiles", a.n, T);
  return COARSE_ERR_INVALID_ARG;
}

}  // namespace coarse
