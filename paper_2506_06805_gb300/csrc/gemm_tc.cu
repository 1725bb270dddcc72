// Tensor-core complex GEMM for sm_103a: tcgen05.mma with TMEM accumulators,
// operands staged by TMA (cp.async.bulk.tensor) into 128-byte-swizzled
// shared memory, mbarrier pipeline, warp-specialised roles.
//
// The complex product is done as ONE real GEMM on an expanded operand:
// A' (2M x 2K) holds rows (Re a, -Im a) and (Im a, Re a) interleaved over k,
// B' (N x 2K) is the interleaved complex B. Rows 2m / 2m+1 of D = A' B'^T are
// then Re / Im of (A B^T)(m, :), i.e. the four real products of the complex
// product ("4M") in a single accumulator tile.
//
// Precision tiers: kind::tf32 with one product (TIER_TF32) or with a hi/lo
// split and three products hi*hi + hi*lo + lo*hi (TIER_TF32X3); kind::f16
// with bf16 hi/lo and three products (TIER_BF16X3); kind::f16 with fp16
// operands scaled by a power of two per operand, one product (TIER_FP16) or
// hi/lo and three (TIER_FP16X3). Accumulation is FP32 in TMEM, promoted to
// FP32 registers every few K blocks; the epilogue accumulates into FP64 (or
// stores FP32 for staging).
//
// CTA layout (320 threads): warps 0-7 epilogue, warp 8 TMA producer, warp 9
// TMEM allocator + MMA issuer; persistent CTAs walk a list of 128 x BN output
// tiles (of up to 16 problems per launch), K optionally split.
// Every mbarrier wait is bounded in time; on expiry the kernel records an
// error flag, drains, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"

namespace cdfns {

namespace {

constexpr int BM = 128;            // real rows per tile (TMEM lanes)
constexpr int ROW_BYTES = 128;     // one swizzle row: 32 fp32 or 64 bf16
constexpr unsigned long long WAIT_NS = 2000000000ull;   // default limit of a pipeline wait (2 s)
constexpr unsigned long long DRAIN_NS = 2000000000ull;  // limit of the waits that drain copies and MMAs

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete: false once
// limit_ns have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// TMEM allocation of one CTA, or (PAIR) the collective allocation of a CTA
// pair: one warp of each CTA executes it and both receive the same address.
template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  if constexpr (PAIR) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  } else {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}
template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  if constexpr (PAIR)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
// --- CTA pairs (clusters of two) ---
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}
// shared::cluster address of the same shared-memory offset in CTA rank 0
__device__ __forceinline__ uint32_t leader_addr(uint32_t a) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"(a));
  return r;
}
// arrive on an mbarrier given by its shared::cluster address
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t a) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on the
// barrier at shared::cluster address bar (the leader's, in a CTA pair)
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar,
                                                 int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1, tile base 1024-byte aligned.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;               // LBO (unused for SW128 K-major)
  d |= static_cast<uint64_t>(1024u >> 4) << 32;       // SBO
  d |= static_cast<uint64_t>(1u) << 46;               // descriptor version
  d |= static_cast<uint64_t>(2u) << 61;               // SWIZZLE_128B
  return d;
}
// Instruction descriptor for kind::tf32 / kind::f16: D f32, A/B K-major.
__host__ __device__ constexpr uint32_t make_idesc(int m, int n, uint32_t ab_type) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}
template <bool BF16, bool PAIR>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if constexpr (PAIR && BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else if constexpr (PAIR) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else if constexpr (BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
// Arrive on bar once the MMAs issued so far have completed: in this CTA, or
// (PAIR) at the same offset in both CTAs of the pair.
template <bool PAIR>
__device__ __forceinline__ void mma_commit_both(uint64_t *bar) {
  if constexpr (PAIR)
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(static_cast<uint16_t>(3))
        : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
// Same, arriving only on the issuing CTA's barrier.
template <bool PAIR>
__device__ __forceinline__ void mma_commit_self(uint64_t *bar) {
  if constexpr (PAIR)
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One GEMM problem of a (possibly grouped) launch. The tensor maps live in
// the kernel parameters (__grid_constant__), 64-byte aligned.
struct alignas(64) TcProblem {
  CUtensorMap mA, mAlo, mB, mBlo;
  long M, N;        // complex rows, columns
  void *C;
  const long *cm, *cn;
  long ldc;
  double2 alpha, beta;
  float2 alpha_f;   // alpha rounded to FP32 (applied to the FP32 tile)
  const float *amax_a, *amax_b;  // FP16 operand scales (nullptr: none)
  float *amax_out;  // TC_OUT_F32: max |written value| x amax_mul (nullptr: none)
  float amax_mul;
  int num_kb;       // K blocks of 128 bytes per row
  int kb_per_split;
  int k_splits, m_tiles, n_tiles;
  int group_m;      // m tiles per raster group (A panels kept in L2)
  int chunk;        // K blocks accumulated in TMEM before promotion
  int out;
  int wmode;        // epilogue write, decided on the host (WM_*): no FP64 tests per element
  int tile_start;   // first index of this problem in the launch's tile space
};
// Epilogue write modes. The FP64 pipe of this GPU retires about two
// operations per SM clock, so the per-element path tests integers only.
enum { WM_F32 = 0, WM_F64_ADD = 1, WM_F64_STORE = 2, WM_F64_BETA = 3 };
constexpr int MAX_PROBLEMS = 16;
struct TcGroup {
  TcProblem p[MAX_PROBLEMS];
  int nprob;
  int total_tiles;
  int *err;
  unsigned long long wait_ns;  // limit of each pipeline wait
};

__device__ __forceinline__ int find_problem(const TcGroup &g, int t) {
  int p = 0;
  while (p + 1 < g.nprob && t >= g.p[p + 1].tile_start) ++p;
  return p;
}

// Local tile index -> (m tile, n tile, k split): groups of group_m m-tiles,
// n-tiles swept inside a group, so a wave of CTAs shares a few A panels and a
// few B panels in L2.
__device__ __forceinline__ void tile_coords(const TcProblem &a, int t, int &m, int &n, int &z) {
  const int mn = a.m_tiles * a.n_tiles;
  z = t / mn;
  const int r0 = t - z * mn;
  const int per_group = a.group_m * a.n_tiles;
  const int g = r0 / per_group;
  const int first_m = g * a.group_m;
  const int gsize = min(a.group_m, a.m_tiles - first_m);
  const int r = r0 - g * per_group;
  m = first_m + r % gsize;
  n = r / gsize;
}

// Persistent CTA (one per SM): warps 0-7 epilogue (TMEM lane quadrant =
// warp % 4, column half = warp / 4), warp 8 TMA producer, warp 9 TMEM
// allocator + MMA issuer, all walking the same tile sequence. TMEM holds two
// accumulator buffers of BN columns. The MMA warp fills one buffer with a
// chunk of `chunk` K blocks while the epilogue warps add the other buffer's
// partial sums into FP32 registers (round to nearest): the tensor core's own
// accumulation only ever spans one chunk, which bounds its truncation bias
// independently of K. Chunk and stage counters run on across tiles, so the
// MMA of the next tile overlaps the epilogue stores of the previous one.
//
// PAIR: the CTAs run as clusters of two on a pair of SMs (tcgen05
// cta_group::2). A work unit is then a 256-row tile: CTA r of the pair loads
// rows [128 r, 128 r + 128) of A and rows [BN/2 r, BN/2 r + BN/2) of B for
// each K block into its own shared memory, both signalling the leader's
// (rank 0) stage barrier; the leader issues M = 256 MMAs that read both
// CTAs' operands (so each SM streams half of B instead of all of it) and
// write each CTA's 128 accumulator rows into that CTA's TMEM; its commits
// arrive on the barriers of both CTAs. Each CTA's epilogue drains its own
// rows and tells the leader, whose TMEM-free barrier counts both CTAs' warps.
// ET: operand type, 0 tf32 (kind::tf32), 1 bf16 / 2 fp16 (kind::f16)
template <int BN, int STAGES, bool SPLIT, int ET, bool PAIR>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_kernel(const __grid_constant__ TcGroup grp) {
  constexpr int A_BYTES = BM * ROW_BYTES;
  constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * ROW_BYTES;  // this CTA's part of B
  constexpr int STAGE_BYTES = (A_BYTES + B_BYTES) * (SPLIT ? 2 : 1);
  constexpr int UNIT_ROWS = PAIR ? 2 * BM : BM;  // real rows per work unit
  constexpr bool F16K = ET != 0;                 // kind::f16 (bf16 or fp16)
  constexpr int K_ELEMS = F16K ? 64 : 32;        // elements per 128-byte row
  constexpr int MMA_K_BYTES = 32;                // K per MMA: 8 tf32 / 16 bf16
  constexpr uint32_t IDESC = make_idesc(UNIT_ROWS, BN, ET == 0 ? 2u : (ET == 1 ? 1u : 0u));
  constexpr int HALF = BN / 2;                   // columns per epilogue warp
  constexpr uint32_t TMEM_COLS = 2 * BN;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;   // [2]
  uint64_t *tempty = tfull + 2;       // [2]
  uint64_t *mdone = tempty + 2;       // every MMA issued has completed
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
  float *stage = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 256);  // 8 x 4 KB

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_units = grp.total_tiles;
  int *const err = grp.err;
  const unsigned long long wait_ns = grp.wait_ns;
  // position of this CTA (pair) in the persistent walk over work units; the
  // special registers are re-read at each use (asm volatile) rather than
  // held live through the loops, which keeps the epilogue warps within their
  // register budget
#define TC_RANK (PAIR ? static_cast<int>(cluster_rank()) : 0)
#define TC_UNIT0 (PAIR ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x))
#define TC_USTEP (PAIR ? static_cast<int>(cluster_count_x()) : static_cast<int>(gridDim.x))

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);   // the (leader's) producer arrival + the bytes of the stage
      mbar_init(&empty[s], 1);  // released by the MMA warp's commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], PAIR ? 16 : 8);  // the epilogue warps (of both CTAs)
    }
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 9) tmem_alloc<PAIR>(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();  // both CTAs' barriers exist before any copy
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 8) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      long it = 0;  // k blocks issued so far (all tiles)
      bool ok = true;
      for (int t = TC_UNIT0; t < n_units && ok; t += TC_USTEP) {
        const TcProblem &P = grp.p[find_problem(grp, t)];
        int m_tile, n_tile, z;
        tile_coords(P, t - P.tile_start, m_tile, n_tile, z);
        const int kb0 = z * P.kb_per_split;
        const int kb1 = min(P.num_kb, kb0 + P.kb_per_split);
        const int ya = m_tile * UNIT_ROWS + TC_RANK * BM;
        const int yb = PAIR ? n_tile * BN + TC_RANK * (BN / 2) : n_tile * BN;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = static_cast<int>(it % STAGES);
          const uint32_t ph = static_cast<uint32_t>(it / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, wait_ns)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          uint8_t *st = smem + s * STAGE_BYTES;
          const int kx = kb * K_ELEMS;
          if constexpr (PAIR) {
            if (TC_RANK == 0) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
            const uint32_t fb = leader_addr(smem_u32(&full[s]));
            tma_load_2d_pair(st, &P.mA, fb, kx, ya);
            tma_load_2d_pair(st + A_BYTES, &P.mB, fb, kx, yb);
            if constexpr (SPLIT) {
              tma_load_2d_pair(st + A_BYTES + B_BYTES, &P.mAlo, fb, kx, ya);
              tma_load_2d_pair(st + 2 * A_BYTES + B_BYTES, &P.mBlo, fb, kx, yb);
            }
          } else {
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(st, &P.mA, &full[s], kx, ya);
            tma_load_2d(st + A_BYTES, &P.mB, &full[s], kx, yb);
            if constexpr (SPLIT) {
              tma_load_2d(st + A_BYTES + B_BYTES, &P.mAlo, &full[s], kx, ya);
              tma_load_2d(st + 2 * A_BYTES + B_BYTES, &P.mBlo, &full[s], kx, yb);
            }
          }
        }
      }
      // the last load issued into each stage must land before the CTA exits
      // (also after an expired wait: no copy may outlive the CTA's shared
      // memory), each with the drain limit; in a pair the leader's barriers
      // count the bytes of both CTAs
      if (TC_RANK == 0) {
        for (long i = (it > STAGES ? it - STAGES : 0); i < it; ++i) {
          if (!mbar_wait(&full[i % STAGES], static_cast<uint32_t>(i / STAGES) & 1u, DRAIN_NS))
            atomicExch(err, 1);
        }
      }
    }
  } else if (warp == 9) {
    if (lane == 0 && TC_RANK == 0) {
      // ---------------- MMA issuer (the leader of a pair) ----------------
      long it = 0;  // k blocks consumed (all tiles)
      long c = 0;   // chunks issued (all tiles)
      bool ok = true;
      for (int t = TC_UNIT0; t < n_units && ok; t += TC_USTEP) {
        const TcProblem &P = grp.p[find_problem(grp, t)];
        int m_tile, n_tile, z;
        tile_coords(P, t - P.tile_start, m_tile, n_tile, z);
        const int kb0 = z * P.kb_per_split;
        const int nkb = min(P.num_kb, kb0 + P.kb_per_split) - kb0;
        const int chunk = P.chunk;
        const int nch = (nkb + chunk - 1) / chunk;
        for (int cc = 0; cc < nch && ok; ++cc, ++c) {
          const int buf = static_cast<int>(c & 1);
          if (c >= 2 && !mbar_wait(&tempty[buf], static_cast<uint32_t>((c - 2) >> 1) & 1u, wait_ns)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + buf * BN;
          const int kend = min(nkb, (cc + 1) * chunk);
          for (int i = 0, kb = cc * chunk; kb < kend; ++i, ++kb, ++it) {
            const int s = static_cast<int>(it % STAGES);
            const uint32_t ph = static_cast<uint32_t>(it / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, wait_ns)) {
              atomicExch(err, 1);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t b0 = a0 + A_BYTES;
            const uint32_t alo = b0 + B_BYTES;
            const uint32_t blo = alo + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < ROW_BYTES / MMA_K_BYTES; ++kk) {
              const uint64_t da = sw128_desc(a0 + kk * MMA_K_BYTES);
              const uint64_t db = sw128_desc(b0 + kk * MMA_K_BYTES);
              mma<F16K, PAIR>(dt, da, db, IDESC, (i > 0 || kk > 0) ? 1u : 0u);
              if constexpr (SPLIT) {
                mma<F16K, PAIR>(dt, da, sw128_desc(blo + kk * MMA_K_BYTES), IDESC, 1u);
                mma<F16K, PAIR>(dt, sw128_desc(alo + kk * MMA_K_BYTES), db, IDESC, 1u);
              }
            }
            mma_commit_both<PAIR>(&empty[s]);
          }
          mma_commit_both<PAIR>(&tfull[buf]);
        }
      }
      // every MMA issued must complete before TMEM is freed (after an
      // expired wait the epilogue no longer waits for them)
      mma_commit_self<PAIR>(mdone);
      if (!mbar_wait(mdone, 0u, DRAIN_NS)) atomicExch(err, 1);
    }
  } else {
    // ---------------- epilogue: 8 warps ----------------
    const int q = warp & 3;
    const int h = warp >> 2;
    long c = 0;
    bool ok = true;
    for (int t = TC_UNIT0; t < n_units && ok; t += TC_USTEP) {
      const TcProblem &args = grp.p[find_problem(grp, t)];
      int m_tile, n_tile, z;
      tile_coords(args, t - args.tile_start, m_tile, n_tile, z);
      const int kb0 = z * args.kb_per_split;
      const int nkb = min(args.num_kb, kb0 + args.kb_per_split) - kb0;
      const int nch = (nkb + args.chunk - 1) / args.chunk;
      float acc[HALF];
#pragma unroll
      for (int j = 0; j < HALF; ++j) acc[j] = 0.f;
      for (int cc = 0; cc < nch; ++cc, ++c) {
        const int buf = static_cast<int>(c & 1);
        if (!mbar_wait(&tfull[buf], static_cast<uint32_t>(c >> 1) & 1u, wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + buf * BN + h * HALF;
#pragma unroll
        for (int j = 0; j < HALF; j += 16) {
          float v[16];
          tmem_ld16(base + j, v);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[j + u] += v[u];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(leader_addr(smem_u32(&tempty[buf])));
          else
            mbar_arrive(&tempty[buf]);
        }
      }
      if (!ok) break;
      // Write-out through a per-warp 32 x 32 float staging block (XOR
      // swizzled, conflict free): lane = TMEM row (Re/Im of complex row
      // lane/2) on the way in, lane = output column on the way out, so each
      // store instruction writes 32 consecutive complex values of one row.
      float *stg = stage + warp * 1024;
      float omax = 0.0f;
      // undo the FP16 operand scales (an exact power of two)
      float usc = 1.0f;
      if (args.amax_a) usc = 1.0f / (fp16_scale(*args.amax_a) * fp16_scale(*args.amax_b));
      // alpha with the scales folded in (exact: usc is a power of two)
      const float2 al = make_float2(usc * args.alpha_f.x, usc * args.alpha_f.y);
      const long nbase = static_cast<long>(n_tile) * BN + h * HALF;
      const long mbase = (static_cast<long>(m_tile) * UNIT_ROWS + TC_RANK * BM) / 2 + q * 16;
      // output row offsets of this warp's 16 complex rows, one per lane,
      // fetched once per tile (the row loop takes them by shuffle)
      long roff = 0;
      if (lane < 16 && mbase + lane < args.M)
        roff = args.cm ? args.cm[mbase + lane] : (mbase + lane) * args.ldc;
#pragma unroll
      for (int j = 0; j < HALF; j += 32) {
#pragma unroll
        for (int u = 0; u < 32; ++u) stg[lane * 32 + (u ^ lane)] = acc[j + u];
        __syncwarp();
        const long n = nbase + j + lane;
        const bool col_ok = n < args.N;
        const long cno = col_ok ? (args.cn ? args.cn[n] : n) : 0;
        const int wm = args.wmode;  // the same for the whole tile
        if (wm == WM_F32) {
          float2 *Cf = reinterpret_cast<float2 *>(args.C);
#pragma unroll 4
          for (int rr = 0; rr < 16; ++rr) {
            const long mc = mbase + rr;
            if (!col_ok || mc >= args.M) continue;
            const float re = usc * stg[(2 * rr) * 32 + (lane ^ (2 * rr))];
            const float im = usc * stg[(2 * rr + 1) * 32 + (lane ^ (2 * rr + 1))];
            Cf[mc * args.ldc + n] = make_float2(re, im);
            omax = fmaxf(omax, fmaxf(fabsf(re), fabsf(im)));
          }
        } else {
          double2 *C = reinterpret_cast<double2 *>(args.C);
#pragma unroll 4
          for (int rr = 0; rr < 16; ++rr) {
            const float sr = stg[(2 * rr) * 32 + (lane ^ (2 * rr))];
            const float si = stg[(2 * rr + 1) * 32 + (lane ^ (2 * rr + 1))];
            const long mc = mbase + rr;
            const long ro = __shfl_sync(0xffffffffu, roff, rr);
            if (!col_ok || mc >= args.M) continue;
            const long off = ro + cno;
            // alpha in FP32 (the product carries FP32 rounding already),
            // widened on the integer pipes; FP64 arithmetic only for a
            // general beta
            const float fr = al.x * sr - al.y * si;
            const float fi = al.x * si + al.y * sr;
            const double xr = f32_to_f64(fr), xi = f32_to_f64(fi);
            if (wm == WM_F64_ADD) {
              // split-K partials, or beta = 1 with one writer per element:
              // the addition runs in L2 (no read round trip, no FP64 work
              // on the SM)
              atomicAdd(&C[off].x, xr);
              atomicAdd(&C[off].y, xi);
            } else if (wm == WM_F64_STORE) {
              C[off] = make_double2(xr, xi);
              omax = fmaxf(omax, fmaxf(fabsf(fr), fabsf(fi)));
            } else {
              const double2 cv = C[off];
              C[off] = make_double2(xr + args.beta.x * cv.x - args.beta.y * cv.y,
                                    xi + args.beta.x * cv.y + args.beta.y * cv.x);
            }
          }
        }
        __syncwarp();
      }
      if (args.amax_out) {
        // largest magnitude written (times amax_mul), for the consumer's FP16 scale
        for (int o = 16; o > 0; o >>= 1) omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, o));
        if (lane == 0)
          atomicMax(reinterpret_cast<unsigned *>(args.amax_out), __float_as_uint(omax * args.amax_mul));
      }
    }
    if (!ok && lane == 0) atomicExch(err, 1);
  }
  tc_fence_before();
  if constexpr (PAIR) {
    // after an expired wait anywhere, let the copies a CTA of the pair may
    // still have in flight into its shared memory land (the leader's stage
    // barriers only track the phases it armed) before either CTA exits
    if (threadIdx.x == 0 && *reinterpret_cast<volatile int *>(err)) {
      const unsigned long long t0 = global_ns();
      while (global_ns() - t0 < 50000000ull) {
      }
    }
  }
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();  // the leader's MMAs into both TMEMs are done
  if (warp == 9) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc<PAIR>(tmem, TMEM_COLS);
  }
#undef TC_RANK
#undef TC_UNIT0
#undef TC_USTEP
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(CC_ERR_CUDA, "cuTensorMapEncodeTiled not found");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// et: 0 fp32 (tf32), 1 bf16, 2 fp16
CUtensorMap make_map(const void *base, long rows, long kp, int box_rows, int et) {
  CUtensorMap m;
  const bool two = et != 0;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(kp) * (two ? 2 : 4)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(two ? 64 : 32),
                             static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = et == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : et == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = get_encoder()(&m, dt,
                             2, const_cast<void *>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(CC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(r));
  return m;
}

// K blocks accumulated in TMEM before promotion to FP32 registers. Each
// promotion makes the epilogue warps drain a buffer, and while they store a
// finished tile they cannot drain the next one's: the MMA then waits once it
// has filled both buffers. Measured on a 4096^3 complex FP16 product: 1110
// TF/s with promotion every 8 K blocks, 1450-1500 with none. The truncation
// bias of the tensor core's FP32 accumulation grows with the chunk (about
// -1e-6 relative per 8 K blocks on same-sign data), so:
//  - one-product tiers (TF32, FP16; rounding ~2^-11 per element): chunks of
//    up to 32 K blocks, and a product whose K range (of one split) has at
//    most 48 K blocks runs as one chunk;
//  - three-product tiers (~2^-22): every 4 K blocks.
// CDFNS_TC_CHUNK (read once) replaces the rule, for tuning.
inline int default_chunk(int tier, int nkb) {
  static const int forced = [] {
    const char *e = std::getenv("CDFNS_TC_CHUNK");
    return e ? std::atoi(e) : 0;
  }();
  if (forced > 0) return forced;
  if (tier_split(tier)) return 4;
  return nkb <= 48 ? std::max(nkb, 1) : 32;
}

template <int BN, int STAGES, bool SPLIT, int ET, bool PAIR>
void launch(const TcDesc *descs, int n, cudaStream_t st, int *err) {
  constexpr int B_ROWS = PAIR ? BN / 2 : BN;     // B rows per CTA and K block
  constexpr int UNIT_ROWS = PAIR ? 2 * BM : BM;  // real rows per work unit
  constexpr int STAGE_BYTES = (BM * ROW_BYTES + B_ROWS * ROW_BYTES) * (SPLIT ? 2 : 1);
  // stages + barrier block (256 B) + 8 warps x 4 KB staging + alignment slack
  constexpr int SMEM = STAGES * STAGE_BYTES + 256 + 8 * 4096 + 1024;
  static_assert((2 * STAGES + 5) * 8 + 8 <= 256, "barrier block");
  static_assert(SMEM <= 232448, "shared memory budget");
  auto kern = tc_gemm_kernel<BN, STAGES, SPLIT, ET, PAIR>;
  // set once per process (thread-safe static initialisation)
  static const bool attr = [&] {
    CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    return true;
  }();
  (void)attr;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  TcGroup grp;
  std::memset(static_cast<void *>(&grp), 0, sizeof(grp));
  long tiles = 0;
  int np = 0;
  for (int q = 0; q < n; ++q) {
    const TcDesc &g = descs[q];
    if (g.M <= 0 || g.N <= 0 || g.Kp <= 0) continue;
    TcProblem &a = grp.p[np++];
    const long mr = 2 * g.M;
    a.mA = make_map(g.A, mr, g.Kp, BM, ET);
    a.mB = make_map(g.B, g.N, g.Kp, B_ROWS, ET);
    a.mAlo = SPLIT ? make_map(g.Alo, mr, g.Kp, BM, ET) : a.mA;
    a.mBlo = SPLIT ? make_map(g.Blo, g.N, g.Kp, B_ROWS, ET) : a.mB;
    a.M = g.M;
    a.N = g.N;
    a.num_kb = static_cast<int>(g.Kp / (ET != 0 ? 64 : 32));
    const int sk = std::max(1, std::min(g.split_k, a.num_kb));
    a.kb_per_split = (a.num_kb + sk - 1) / sk;
    a.k_splits = (a.num_kb + a.kb_per_split - 1) / a.kb_per_split;
    a.m_tiles = static_cast<int>((mr + UNIT_ROWS - 1) / UNIT_ROWS);
    a.n_tiles = static_cast<int>((g.N + BN - 1) / BN);
    // raster groups: as many A panels (a unit's rows x the K range of a
    // split) as fit in ~24 MB of L2 share each B panel while it is resident
    const double panel = static_cast<double>(UNIT_ROWS) * a.kb_per_split * ROW_BYTES * (SPLIT ? 2 : 1);
    a.group_m = g.group_m > 0 ? std::min(g.group_m, a.m_tiles)
                              : static_cast<int>(std::max(1.0, std::min<double>(a.m_tiles, 24.0e6 / panel)));
    a.chunk = g.chunk > 0 ? g.chunk : default_chunk(g.tier, a.kb_per_split);
    a.out = g.out;
    a.wmode = g.out == TC_OUT_F32 ? WM_F32
              : g.out == TC_OUT_F64_ATOMIC ? WM_F64_ADD
              : (g.beta.x == 0.0 && g.beta.y == 0.0) ? WM_F64_STORE
              : (g.beta.x == 1.0 && g.beta.y == 0.0) ? WM_F64_ADD
                                                     : WM_F64_BETA;
    a.C = g.C;
    a.cm = g.cm;
    a.cn = g.cn;
    a.ldc = g.ldc;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.alpha_f = make_float2(static_cast<float>(g.alpha.x), static_cast<float>(g.alpha.y));
    a.amax_a = g.amax_a;
    a.amax_b = g.amax_b;
    const bool plain = g.out == TC_OUT_F64 && g.beta.x == 0.0 && g.beta.y == 0.0;
    if (g.amax_out && g.out != TC_OUT_F32 && !plain)
      fail(CC_ERR_ARG, "gemm_tc: output maxima need plain stores (F32, or F64 with beta = 0)");
    a.amax_out = g.amax_out;
    a.amax_mul = g.amax_mul;
    if ((g.amax_a == nullptr) != (g.amax_b == nullptr))
      fail(CC_ERR_ARG, "gemm_tc: FP16 operand scales come in pairs");
    a.tile_start = static_cast<int>(tiles);
    tiles += static_cast<long>(a.m_tiles) * a.n_tiles * a.k_splits;
    if (tiles > 0x7fffffffL) fail(CC_ERR_ARG, "gemm_tc: too many tiles");
  }
  if (np == 0) return;
  grp.nprob = np;
  grp.total_tiles = static_cast<int>(tiles);
  grp.err = err;
  grp.wait_ns = tc_wait_limit();
  if constexpr (!PAIR) {
    dim3 grid(static_cast<unsigned>(std::min<long>(tiles, sms)));
    kern<<<grid, 320, SMEM, st>>>(grp);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // persistent pairs: as many clusters as can be resident at once
    static const int max_clusters = [&] {
      int mc = 0;
      cfg.gridDim = dim3(static_cast<unsigned>(2 * (sms / 2)));
      CUDA_CHECK(cudaOccupancyMaxActiveClusters(&mc, kern, &cfg));
      if (mc < 1) fail(CC_ERR_UNSUPPORTED, "gemm_tc: no resident CTA pair");
      return mc;
    }();
    cfg.gridDim = dim3(static_cast<unsigned>(2 * std::min<long>(tiles, max_clusters)));
    CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, grp));
  }
  LAUNCH_CHECK();
  count_launch();
}

void check_desc(const TcDesc &g) {
  if (g.Kp % tc_k_align(g.tier)) fail(CC_ERR_ARG, "gemm_tc: Kp not padded");
  if ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(g.B)) & 15)
    fail(CC_ERR_ARG, "gemm_tc: operands must be 16-byte aligned");
}

// CTA pairs (cta_group::2) for wide tiles: on unless CDFNS_PAIR is "0"
// (read once), and used when the launch has enough 256-row units to give
// every SM pair one and padding the rows to 256 instead of 128 adds less
// than 3 % to the tensor work.
bool pair_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("CDFNS_PAIR");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool pair_pays(const TcDesc *d, int n) {
  long units = 0;
  double rows1 = 0, rows2 = 0;
  for (int q = 0; q < n; ++q) {
    if (d[q].M <= 0 || d[q].N <= 0) continue;
    const long r = 2 * d[q].M, nt = (d[q].N + 255) / 256;
    units += ((r + 255) / 256) * nt;
    rows1 += static_cast<double>((r + 127) / 128 * 128) * nt;
    rows2 += static_cast<double>((r + 255) / 256 * 256) * nt;
  }
  return units >= 76 && rows2 <= 1.03 * rows1;
}

void dispatch(const TcDesc *d, int n, bool wide, cudaStream_t st, int *err) {
  const bool pair = wide && pair_enabled() && pair_pays(d, n);
  switch (d[0].tier) {
    case TIER_TF32:
      if (pair) launch<256, 6, false, 0, true>(d, n, st, err);
      else if (wide) launch<256, 4, false, 0, false>(d, n, st, err);
      else launch<128, 6, false, 0, false>(d, n, st, err);
      break;
    case TIER_TF32X3:
      if (pair) launch<256, 3, true, 0, true>(d, n, st, err);
      else if (wide) launch<256, 2, true, 0, false>(d, n, st, err);
      else launch<128, 3, true, 0, false>(d, n, st, err);
      break;
    case TIER_BF16X3:
      if (pair) launch<256, 3, true, 1, true>(d, n, st, err);
      else if (wide) launch<256, 2, true, 1, false>(d, n, st, err);
      else launch<128, 3, true, 1, false>(d, n, st, err);
      break;
    case TIER_FP16:
      if (pair) launch<256, 6, false, 2, true>(d, n, st, err);
      else if (wide) launch<256, 4, false, 2, false>(d, n, st, err);
      else launch<128, 6, false, 2, false>(d, n, st, err);
      break;
    case TIER_FP16X3:
      if (pair) launch<256, 3, true, 2, true>(d, n, st, err);
      else if (wide) launch<256, 2, true, 2, false>(d, n, st, err);
      else launch<128, 3, true, 2, false>(d, n, st, err);
      break;
    default:
      fail(CC_ERR_ARG, "gemm_tc: bad tier");
  }
}

}  // namespace

namespace {
std::atomic<unsigned long long> g_wait_ns{0};
}  // namespace

void tc_set_wait_limit(unsigned long long ns) { g_wait_ns.store(ns); }
unsigned long long tc_wait_limit() {
  const unsigned long long ns = g_wait_ns.load();
  return ns ? ns : WAIT_NS;
}

int tc_k_align(int tier) { return tier_half(tier) ? 64 : 32; }

int tc_pick_bn(long N) {
  const double u256 = static_cast<double>(N) / (((N + 255) / 256) * 256);
  const double u128 = static_cast<double>(N) / (((N + 127) / 128) * 128);
  return u128 > u256 + 0.08 ? 128 : 256;
}

int tc_pick_split(long tiles, long nkb, int num_sms) {
  int sk = 1;
  if (tiles <= 0 || tiles >= 8L * num_sms || nkb < 8) return sk;
  const long P = num_sms;
  // a handful of tiles over a long K: one split per free SM
  if (tiles * 32 < P) return static_cast<int>(std::max<long>(1, std::min<long>(nkb / 4, P / tiles)));
  auto eff = [&](long sp) {
    const long tt = tiles * sp;
    return static_cast<double>(tt) / (static_cast<double>((tt + P - 1) / P) * P);
  };
  // a split turns every output write into atomic additions in L2 (and the
  // output into a read-modify-write in DRAM): only worth it for a clear
  // gain in wave occupancy
  double best = eff(1);
  const double need = tiles < 2L * P ? 0.02 : 0.15;
  const long smax = std::min<long>(32, nkb / 4);
  for (long sp = 2; sp <= smax; ++sp) {
    const double e = eff(sp) * (1.0 - 0.005 * static_cast<double>(sp - 1));
    if (e > best + need) {
      best = e;
      sk = static_cast<int>(sp);
    }
  }
  return sk;
}
size_t tc_elem_bytes(int tier) { return tier_half(tier) ? 2 : 4; }

// ---------------------------------------------------------------------------
// Autotuner: per (tier, shape bucket) the tile width, raster group and TMEM
// promotion chunk are chosen by timing a few candidates once, on a scratch
// FP32 output, when CDFNS_AUTOTUNE=1. Choices persist in the JSON file named
// by CDFNS_TUNE_CACHE ({"key": [bn, group_m, chunk], ...}). Never runs while
// the stream is being captured.
// ---------------------------------------------------------------------------
namespace {

struct Choice {
  int bn, group_m, chunk;
};
std::mutex g_tune_mu;
std::map<std::string, Choice> g_tune;
bool g_tune_loaded = false;

long pow2_up(long x) {
  long p = 1;
  while (p < x) p <<= 1;
  return p;
}

std::string tune_key(const TcDesc &g) {
  return std::to_string(g.tier) + ":" + std::to_string(pow2_up(2 * g.M)) + "x" +
         std::to_string(pow2_up(g.N)) + "x" + std::to_string(pow2_up(g.Kp)) + ":" +
         std::to_string(g.split_k > 1);
}

const char *tune_path() { return std::getenv("CDFNS_TUNE_CACHE"); }
bool tune_enabled() {
  const char *e = std::getenv("CDFNS_AUTOTUNE");
  return e && e[0] == '1';
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *p = tune_path();
  if (!p) return;
  FILE *f = std::fopen(p, "r");
  if (!f) return;
  char key[256];
  int bn, gm, ch;
  // format written by tune_save: one "key": [bn, group_m, chunk] per line
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    if (std::sscanf(line, " \"%255[^\"]\": [%d, %d, %d]", key, &bn, &gm, &ch) == 4)
      g_tune[key] = Choice{bn, gm, ch};
  }
  std::fclose(f);
}

void tune_save() {
  const char *p = tune_path();
  if (!p) return;
  FILE *f = std::fopen(p, "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto &kv : g_tune) {
    std::fprintf(f, "  \"%s\": [%d, %d, %d]%s\n", kv.first.c_str(), kv.second.bn, kv.second.group_m,
                 kv.second.chunk, ++i < g_tune.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  std::fclose(f);
}

Choice tune(const TcDesc &g, cudaStream_t st, int *err) {
  const int dch = default_chunk(g.tier, static_cast<int>(g.Kp / (tier_half(g.tier) ? 64 : 32)));
  const Choice cands[] = {{256, 0, dch}, {256, 1, dch}, {256, 16, dch},
                          {128, 0, dch}, {256, 0, 2 * dch}, {128, 1, dch}};
  void *scratch = nullptr;
  CUDA_CHECK(cudaMalloc(&scratch, sizeof(float2) * g.M * g.N));
  cudaEvent_t e0, e1;
  CUDA_CHECK(cudaEventCreate(&e0));
  CUDA_CHECK(cudaEventCreate(&e1));
  Choice best = cands[0];
  float best_ms = 1e30f;
  for (const Choice &c : cands) {
    TcDesc t = g;
    t.out = TC_OUT_F32;
    t.C = scratch;
    t.cm = t.cn = nullptr;
    t.ldc = g.N;
    t.bn = c.bn;
    t.group_m = c.group_m;
    t.chunk = c.chunk;
    dispatch(&t, 1, c.bn == 256, st, err);  // warm
    CUDA_CHECK(cudaEventRecord(e0, st));
    dispatch(&t, 1, c.bn == 256, st, err);
    CUDA_CHECK(cudaEventRecord(e1, st));
    CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0;
    CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  return best;
}

}  // namespace

void gemm_tc(const TcDesc &g0, cudaStream_t st, int *err) {
  if (g0.M <= 0 || g0.N <= 0 || g0.Kp <= 0) return;
  check_desc(g0);
  TcDesc g = g0;
  if (tune_enabled() || tune_path()) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    const std::string key = tune_key(g);
    auto it = g_tune.find(key);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (it == g_tune.end() && tune_enabled() && !g.no_tune && cap == cudaStreamCaptureStatusNone) {
      g_tune[key] = tune(g, st, err);
      tune_save();
      it = g_tune.find(key);
    }
    if (it != g_tune.end()) {
      g.bn = it->second.bn;
      g.group_m = it->second.group_m;
      g.chunk = it->second.chunk;
    }
  }
  const bool wide = g.bn > 0 ? g.bn == 256 : g.N >= 192;
  dispatch(&g, 1, wide, st, err);
}

void gemm_tc_grouped(const std::vector<TcDesc> &descs, cudaStream_t st, int *err) {
  // one launch per (tier, width) class, at most MAX_PROBLEMS problems each
  for (int tier = TIER_TF32; tier <= TIER_LAST; ++tier) {
    for (int w = 0; w < 2; ++w) {
      std::vector<TcDesc> cls;
      for (const TcDesc &g : descs) {
        if (g.tier != tier || g.M <= 0 || g.N <= 0 || g.Kp <= 0) continue;
        const bool wide = g.bn > 0 ? g.bn == 256 : g.N >= 192;
        if (wide != (w == 1)) continue;
        check_desc(g);
        cls.push_back(g);
      }
      for (size_t k = 0; k < cls.size(); k += MAX_PROBLEMS) {
        const int n = static_cast<int>(std::min<size_t>(MAX_PROBLEMS, cls.size() - k));
        dispatch(cls.data() + k, n, w == 1, st, err);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Operand packing (FP64 complex -> expanded real planes)
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Two adjacent elements (idx even) as one 8-byte (fp32) or 4-byte (bf16,
// fp16) store. PT: 0 tf32 hi (+ lo), 1 bf16 hi (+ lo), 2 fp16 of sc * x,
// 3 fp16 hi + lo of sc * x.
template <int PT>
__device__ __forceinline__ void split_store2(void *hi, void *lo, long idx, float x, float y,
                                             float sc) {
  if constexpr (PT == 1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    reinterpret_cast<__nv_bfloat162 *>(hi)[idx >> 1] = h;
    if (lo) {
      const float2 hf = __bfloat1622float2(h);
      reinterpret_cast<__nv_bfloat162 *>(lo)[idx >> 1] = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    }
  } else if constexpr (PT == 2 || PT == 3) {
    const float sx = sc * x, sy = sc * y;
    const __half2 h = __floats2half2_rn(sx, sy);
    reinterpret_cast<__half2 *>(hi)[idx >> 1] = h;
    if (PT == 3 && lo) {
      const float2 hf = __half22float2(h);
      reinterpret_cast<__half2 *>(lo)[idx >> 1] = __floats2half2_rn(sx - hf.x, sy - hf.y);
    }
  } else {
    const float hx = to_tf32(x), hy = to_tf32(y);
    reinterpret_cast<float2 *>(hi)[idx >> 1] = make_float2(hx, hy);
    if (lo) reinterpret_cast<float2 *>(lo)[idx >> 1] = make_float2(to_tf32(x - hx), to_tf32(y - hy));
  }
}

template <int PT, bool EXPAND>
__device__ __forceinline__ void pack_store(void *hi, void *lo, long r, long kc, long Kp, double2 a,
                                           bool conj, float sc) {
  const float re = f64_to_f32(a.x), im = conj ? -f64_to_f32(a.y) : f64_to_f32(a.y);
  if (EXPAND) {
    split_store2<PT>(hi, lo, (2 * r) * Kp + 2 * kc, re, -im, sc);
    split_store2<PT>(hi, lo, (2 * r + 1) * Kp + 2 * kc, im, re, sc);
  } else {
    split_store2<PT>(hi, lo, r * Kp + 2 * kc, re, im, sc);
  }
}

// Block (BX, BY): x over complex k (padded to Kp/2), y over rows
// (grid-stride); BX shrinks to the row length so short rows keep every
// thread busy.
template <int PT, bool EXPAND>
__global__ void __launch_bounds__(256) pack_kernel(const double2 *__restrict__ src,
                                                   const long *__restrict__ rt,
                                                   const long *__restrict__ kt, long ld, bool conj,
                                                   long rows, long K, long Kp, void *hi, void *lo,
                                                   const float *amax) {
  const long kc = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;  // complex k
  if (kc >= Kp / 2) return;
  const float sc = (PT >= 2 && amax) ? fp16_scale(*amax) : 1.0f;
  const long kof = kc < K ? (kt ? kt[kc] : kc) : 0;
  const long step = static_cast<long>(gridDim.y) * blockDim.y;
  // four rows per pass: their loads are all in flight before the stores
  for (long r = blockIdx.y * static_cast<long>(blockDim.y) + threadIdx.y; r < rows; r += 4 * step) {
    double2 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long ru = r + u * step;
      a[u] = make_double2(0.0, 0.0);
      if (kc < K && ru < rows) a[u] = src[(rt ? rt[ru] : ru * ld) + kof];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long ru = r + u * step;
      if (ru < rows) pack_store<PT, EXPAND>(hi, lo, ru, kc, Kp, a[u], conj, sc);
    }
  }
}

// Rows (mostly) contiguous in the source (unit stride or a table whose
// neighbouring entries are neighbours; k through a table or a large
// stride): 32 x 32 tiles transposed through shared memory so that the loads
// run along rows and the stores along k. Block (32, 8).
template <int PT, bool EXPAND>
__global__ void __launch_bounds__(256) pack_t_kernel(const double2 *__restrict__ src,
                                                     const long *__restrict__ rt, long ld,
                                                     const long *__restrict__ kt, bool conj,
                                                     long rows, long K, long Kp, void *hi,
                                                     void *lo, const float *amax) {
  __shared__ double2 tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float sc = (PT >= 2 && amax) ? fp16_scale(*amax) : 1.0f;
  const long k0 = blockIdx.x * 32L;
  for (long r0 = blockIdx.y * 32L; r0 < rows; r0 += gridDim.y * 32L) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long k = k0 + ty + 8 * j, r = r0 + tx;
      double2 a = make_double2(0.0, 0.0);
      if (k < K && r < rows) a = src[(rt ? rt[r] : r * ld) + (kt ? kt[k] : k)];
      tile[ty + 8 * j][tx] = a;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long r = r0 + ty + 8 * j, kc = k0 + tx;
      if (r < rows && kc < Kp / 2)
        pack_store<PT, EXPAND>(hi, lo, r, kc, Kp, tile[tx][ty + 8 * j], conj, sc);
    }
    __syncthreads();
  }
}

// max(|Re|, |Im|) over a table-addressed operand; block maxima combined
// with an unsigned atomicMax on the float bits (non-negative floats order
// like their bit patterns).
__device__ __forceinline__ void block_max_store(float m, float *amax) {
  __shared__ float sh[8];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int w = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  if (l == 0) sh[w] = m;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float x = 0.0f;
    const int nw = static_cast<int>(blockDim.x * blockDim.y) >> 5;
    for (int i = 0; i < nw; ++i) x = fmaxf(x, sh[i]);
    atomicMax(reinterpret_cast<unsigned *>(amax), __float_as_uint(x));
  }
}

// Block (BX, BY): x along the operand's contiguous direction (rows when
// rows_inner, else k), y along the other; both grid-stride.
__global__ void __launch_bounds__(256) absmax_kernel(const double2 *__restrict__ src,
                                                     const long *__restrict__ rt,
                                                     const long *__restrict__ kt, long ld,
                                                     long rows, long K, bool rows_inner,
                                                     float *amax) {
  float m = 0.0f;
  const long X = rows_inner ? rows : K, Y = rows_inner ? K : rows;
  const long xstep = static_cast<long>(gridDim.x) * blockDim.x;
  const long ystep = static_cast<long>(gridDim.y) * blockDim.y;
  for (long xi = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; xi < X; xi += xstep) {
    // four elements per pass, loads in flight together
    for (long yi = blockIdx.y * static_cast<long>(blockDim.y) + threadIdx.y; yi < Y; yi += 4 * ystep) {
      double2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long yu = yi + u * ystep;
        const long r = rows_inner ? xi : yu, k = rows_inner ? yu : xi;
        a[u] = yu < Y ? src[(rt ? rt[r] : r * ld) + (kt ? kt[k] : k)] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        m = fmaxf(m, fmaxf(fabsf(f64_to_f32(a[u].x)), fabsf(f64_to_f32(a[u].y))));
    }
  }
  block_max_store(m, amax);
}

// Contiguous operand: four independent 16-byte loads per thread in flight.
__global__ void __launch_bounds__(256) absmax_flat_kernel(const double2 *__restrict__ src, long n,
                                                          float *amax) {
  float m = 0.0f;
  const long step = static_cast<long>(gridDim.x) * blockDim.x;
  long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
  for (; i + 3 * step < n; i += 4 * step) {
    double2 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = src[i + u * step];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      m = fmaxf(m, fmaxf(fabsf(f64_to_f32(a[u].x)), fabsf(f64_to_f32(a[u].y))));
  }
  for (; i < n; i += step) {
    const double2 a = src[i];
    m = fmaxf(m, fmaxf(fabsf(f64_to_f32(a.x)), fabsf(f64_to_f32(a.y))));
  }
  block_max_store(m, amax);
}

template <bool EXPAND>
void pack_launch(const cplx *src, const long *rt, const long *kt, long ld, bool conj, long rows,
                 long K, long Kp, int tier, void *hi, void *lo, cudaStream_t st,
                 const float *amax, bool rows_unit) {
  if (rows <= 0) return;
  void *l = tier_split(tier) ? lo : nullptr;
  const int pt = tier == TIER_BF16X3 ? 1 : (tier == TIER_FP16 ? 2 : (tier == TIER_FP16X3 ? 3 : 0));
  const long kh = Kp / 2;
  if (kt && rows > 1 && K > 1 && ((!rt && ld == 1) || rows_unit)) {
    dim3 block(32, 8);
    dim3 grid(static_cast<unsigned>((kh + 31) / 32),
              static_cast<unsigned>(std::min<long>((rows + 31) / 32, 65535)));
    switch (pt) {
      case 1: pack_t_kernel<1, EXPAND><<<grid, block, 0, st>>>(src, rt, ld, kt, conj, rows, K, Kp, hi, l, amax); break;
      case 2: pack_t_kernel<2, EXPAND><<<grid, block, 0, st>>>(src, rt, ld, kt, conj, rows, K, Kp, hi, l, amax); break;
      case 3: pack_t_kernel<3, EXPAND><<<grid, block, 0, st>>>(src, rt, ld, kt, conj, rows, K, Kp, hi, l, amax); break;
      default: pack_t_kernel<0, EXPAND><<<grid, block, 0, st>>>(src, rt, ld, kt, conj, rows, K, Kp, hi, l, amax);
    }
  } else {
    // x over complex k: as few 32-wide groups per block row as cover it in
    // ceil(kh / 256) blocks, so a short K leaves few threads idle
    const long nbx = (kh + 255) / 256;
    const int bx = static_cast<int>(32 * (((kh + 31) / 32 + nbx - 1) / nbx));
    const int by = std::max(1, 256 / bx);
    dim3 block(bx, by);
    // four rows per thread when there are blocks enough to fill the GPU
    const long gx = (kh + bx - 1) / bx;
    const long rpt = gx * ((rows + 4L * by - 1) / (4L * by)) >= 8L * 152 ? 4 : 1;
    dim3 grid(static_cast<unsigned>(gx),
              static_cast<unsigned>(std::min<long>((rows + rpt * by - 1) / (rpt * by), 65535)));
    switch (pt) {
      case 1: pack_kernel<1, EXPAND><<<grid, block, 0, st>>>(src, rt, kt, ld, conj, rows, K, Kp, hi, l, amax); break;
      case 2: pack_kernel<2, EXPAND><<<grid, block, 0, st>>>(src, rt, kt, ld, conj, rows, K, Kp, hi, l, amax); break;
      case 3: pack_kernel<3, EXPAND><<<grid, block, 0, st>>>(src, rt, kt, ld, conj, rows, K, Kp, hi, l, amax); break;
      default: pack_kernel<0, EXPAND><<<grid, block, 0, st>>>(src, rt, kt, ld, conj, rows, K, Kp, hi, l, amax);
    }
  }
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace

void tc_pack_A(const cplx *src, const long *am, const long *ak, long lda, bool conj, long M,
               long K, long Kp, int tier, void *hi, void *lo, cudaStream_t st, const float *amax,
               bool rows_unit) {
  if (tier_scaled(tier) && !amax) fail(CC_ERR_ARG, "tc_pack_A: FP16 planes need amax");
  pack_launch<true>(src, am, ak, lda, conj, M, K, Kp, tier, hi, lo, st, amax, rows_unit);
}
void tc_pack_B(const cplx *src, const long *bn, const long *bk, long ldb, bool conj, long N,
               long K, long Kp, int tier, void *hi, void *lo, cudaStream_t st, const float *amax,
               bool rows_unit) {
  if (tier_scaled(tier) && !amax) fail(CC_ERR_ARG, "tc_pack_B: FP16 planes need amax");
  pack_launch<false>(src, bn, bk, ldb, conj, N, K, Kp, tier, hi, lo, st, amax, rows_unit);
}

void tc_absmax(const cplx *src, const long *rt, const long *kt, long ld, long rows, long K,
               float *amax, cudaStream_t st) {
  CUDA_CHECK(cudaMemsetAsync(amax, 0, sizeof(float), st));
  if (rows <= 0 || K <= 0) return;
  if (!rt && !kt && (rows == 1 || ld == K)) {
    // one contiguous block of rows * K elements
    const long n = rows * K;
    const long blocks = std::max<long>(1, std::min<long>((n + 1023) / 1024, 152L * 8));
    absmax_flat_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(src, n, amax);
    LAUNCH_CHECK();
    count_launch();
    return;
  }
  const bool rows_inner = !rt && ld == 1;  // unit row stride: sweep rows fastest
  const long X = rows_inner ? rows : K, Y = rows_inner ? K : rows;
  const int bx = static_cast<int>(std::min<long>(256, std::max<long>(32, (X + 31) / 32 * 32)));
  const int by = 256 / bx;
  // at most ~16 blocks per SM in all: threads stride over the operand
  const long gx = std::min<long>((X + bx - 1) / bx, 152L * 16);
  const long gy = std::max<long>(
      1, std::min<long>(std::min<long>((Y + by - 1) / by, 65535L), std::max<long>(1, 152L * 16 / gx)));
  absmax_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), dim3(bx, by), 0, st>>>(
      src, rt, kt, ld, rows, K, rows_inner, amax);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace cdfns
