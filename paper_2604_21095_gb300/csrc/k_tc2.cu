// Tensor-core scan on CTA pairs: Eq. 2 of Section 2.2 with tcgen05.mma.cta_group::2.
//
// The same product as k_tc.cu, D = A (B_hi + B_lo)^T + c (sum_i B), on 256 x 256 tiles
// computed by a cluster of two CTAs on two SMs. Each CTA loads its own 128 marker rows of A
// and its own half (128 phenotype rows) of B_hi / B_lo; the pair's leader (cluster rank 0)
// issues one 256 x 256 x 16 MMA that reads A from both CTAs and B from both CTAs and writes
// rows 0-127 of D into the leader's tensor memory and rows 128-255 into the peer's. Per SM,
// each MMA of the same size reads 8 KB of shared memory instead of 12 KB, and each K block
// brings 24 KB over L2 instead of 40 KB, which is what limits the one-CTA kernel.
//
// Roles (384 threads, three warpgroups, as in k_tc.cu):
//   warp 0 lane 0 (both CTAs)   TMA producer into the local stage ring; every copy signals
//                               the leader's full barrier (cta_group::2 completion). The
//                               leader's producer also takes the pair's next tile (next_tile)
//                               and publishes its index to every role of both CTAs
//   warp 1 lane 0 (leader only) MMA issuer; commits are multicast to both CTAs' barriers
//   warps 4..11 (both CTAs)     epilogue on the local 128 rows; the drained signal goes to
//                               the leader's chunk-empty barrier (16 arrivals: 8 per CTA)
//   warps 2, 3 (both CTAs)      with packed genotypes (OPA_2BIT / OPA_U8): decoders of the
//                               local 128 A rows (tc_common.cuh); each warp arrives once on the
//                               leader's full barrier after its stores
// Accumulation is chunked as in k_tc.cu (a fresh accumulator every 1024 samples, FP32 totals in
// registers) when every statistic is written, every 2048 samples when only hits and best markers
// are kept (chunk_kb). Every wait is bounded; a timeout raises the abort flag in both CTAs.
#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace tg {
namespace {

using namespace tcx;

constexpr int HB_BYTES = 128 * TBK * 2;  // one CTA's half of a B tile: 8 KB

// K blocks per stage: two with the decoded operand, so that each row's two consecutive 64-byte
// segments are requested back to back (better DRAM page use where the kernel streams HBM, at
// small P); one when the A tiles are decoded here.
template <int OPA>
constexpr int kStageKB = OPA == OPA_TMA ? 2 : 1;

template <int OPA>
struct Cfg2 {
  // per K block: A, this CTA's halves of B_hi and B_lo (24 KB); when decoding here, plus the
  // CTA's packed rows (2 or 4 KB)
  static constexpr int KS = kStageKB<OPA>;
  static constexpr int kStageBytes = KS * (A_BYTES + 2 * HB_BYTES) + DecCfg<OPA>::kPackBytes;
  static constexpr int kStages = 8 / KS;
  static constexpr int kBarBytes = 512;
  static constexpr int kSmem = kStages * kStageBytes + kBarBytes + 1024;
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

// Tile indices pass from the leader's producer to every other role of both CTAs through a
// ring of kTileRing shared-memory slots (a full barrier per slot in each CTA, an empty
// barrier per slot in the leader).
constexpr int kTileRing = 4;

constexpr uint32_t kIdesc2 = idesc_bf16_m(256, 256);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t num_clusters() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// TMA into local shared memory, completion counted on a barrier that may be the peer's.
__device__ __forceinline__ void tma_load_2d_pair(const CUtensorMap* map, uint32_t dst,
                                                 uint32_t bar_cluster, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void tc2_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc2), "r"(accumulate)
      : "memory");
}
// Arrive on the barrier at this offset in both CTAs once every prior MMA has completed.
__device__ __forceinline__ void tc2_commit_both(uint32_t bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void tc2_commit_local(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// Tile order and soft lockstep of the CTA pairs. The tiles in flight at once share their A rows
// and panel columns through L2 only while they stream the same K range at about the same time;
// pairs that drift apart read their slabs from DRAM again (4x the traffic, and the power, at
// full size). With a counter (zeroed per launch), a pair takes the next tile of the raster
// when it is ready for one, and starts loading it once all but kLockstepSlack tiles of that
// tile's wave (the ncl tiles in flight together) have been taken, or after kLockstepNs: a pair
// that runs slower than the others takes fewer tiles instead of holding every wave back (with
// a fixed order, pair c taking every ncl-th tile, the last pair to start set the pace of every
// wave), and a pair that is not resident delays the others by at most the time limit and never
// causes an error. Without a counter, pair c takes tiles c, c + ncl, c + 2 ncl, ... without
// waiting. Indices past the last tile (returned as num_tiles) end the pair's work.
constexpr long long kLockstepNs = 30000;
constexpr int kLockstepSlack = 2;
__device__ __forceinline__ int next_tile(unsigned long long* ctr, int i, int cid, int ncl,
                                         int num_tiles) {
  if (!ctr) return min(cid + i * ncl, num_tiles);
  const unsigned long long t = atomicAdd(ctr, 1ull);
  if (t >= (unsigned long long)num_tiles) return num_tiles;
  const long long need = min((long long)num_tiles,
                             (long long)(t / ncl + 1) * ncl - kLockstepSlack);
  const uint64_t t0 = globaltimer_ns();
  while ((long long)*reinterpret_cast<volatile unsigned long long*>(ctr) < need) {
    if ((long long)(globaltimer_ns() - t0) > kLockstepNs) break;
    __nanosleep(64);
  }
  return (int)t;
}

// Accumulation chunks (K blocks per fresh accumulator): kChunkKB (1,024 samples) when every
// statistic is written (FULL), twice that when the launch keeps only hits and per-phenotype
// best markers. There the products only decide which pairs pass the threshold and which marker
// ranks first, and every reported statistic of a hit is recomputed in FP64 from the genotypes
// (k_hit_stats); half the chunk drains take 3% off the launch, and the FP32 error of the
// totals stays within the r tolerance (the best keys) and far inside the threshold band.
__device__ __forceinline__ int chunk_kb(const EpiParams& ep) {
  return ep.do_full ? kChunkKB : 2 * kChunkKB;
}
__device__ __forceinline__ int chunk_end_c(int kb0, int num_kb, int ckb) {
  const int e = kb0 == 0 ? kFirstChunks * ckb : kb0 + ckb;
  return e < num_kb ? e : num_kb;
}

// K direction of a tile: the tiles of odd waves stream K from the end. A wave reads about
// 300 MB of A rows and panel columns at the bench's sizes, more than L2 holds, so a wave that
// starts where the previous one ended finds the last-streamed slabs (chiefly the A rows of the
// raster group's m-tile pairs, which consecutive waves share) still in L2 instead of fetching
// them from DRAM again. Only the order of the FP32 chunk sums changes; every tile still adds
// the same K blocks in chunks of the same sizes.
__device__ __forceinline__ bool k_reversed(int tile, int ncl) { return ((tile / ncl) & 1) != 0; }

// mbarrier wait with acquire at cluster scope (the phase may be completed by the other CTA),
// bounded like mbar_wait.
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity,
                                                  volatile int* abort_flag, long long limit_ns,
                                                  uint32_t* status) {
  if (mbar_try_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)
      if (mbar_try_cluster(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((long long)(globaltimer_ns() - t0) > limit_ns) {
      *abort_flag = 1;
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
}

// Tile (pair of m-tiles, n-tile) of cluster-level tile index `tile`; group_p m-tile pairs
// per raster group.
__device__ __forceinline__ void tile_coord2(int tile, int n_mp, int n_nt, int group_p, int& mp,
                                            int& nt) {
  const int group = group_p * n_nt;
  const int g = tile / group;
  const int first = g * group_p;
  const int gm = min(group_p, n_mp - first);
  const int idx = tile - g * group;
  mp = first + idx % gm;
  nt = idx / gm;
}

template <int OPA>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_tc2_scan(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmBhi,
               const __grid_constant__ CUtensorMap tmBlo, int num_kb, int n_mt, int n_nt,
               int group_p, long long spin_ns, EpiParams ep,
              const __grid_constant__ DecodeArgs da) {
  using C = Cfg2<OPA>;
  constexpr bool kFused = OPA != OPA_TMA;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t bars = base + S * C::kStageBytes;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (S + s); };
  auto cfull_bar = [&](int a) { return bars + 8u * (2 * S + a); };
  auto cempty_bar = [&](int a) { return bars + 8u * (2 * S + 2 + a); };
  const uint32_t drain_bar = bars + 8u * (2 * S + 4);
  auto pfull_bar = [&](int s) { return bars + 8u * (2 * S + 5 + s); };  // local packed rows landed
  auto tfull_bar = [&](int r) { return bars + 8u * (3 * S + 5 + r); };   // tile slot written
  auto tempty_bar = [&](int r) { return bars + 8u * (3 * S + 5 + kTileRing + r); };  // leader's
  constexpr int kBarEnd = 8 * (3 * S + 5 + 2 * kTileRing);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * C::kStageBytes + kBarEnd);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* tile_slot = reinterpret_cast<volatile int*>(tmem_slot + 2);
  static_assert(kBarEnd + 8 + 4 * kTileRing <= C::kBarBytes, "barrier area");
  // consumers of each tile slot: the leader's MMA thread, the peer's producer, the epilogue
  // warps of both CTAs and, when decoding here, the decoder warps of both CTAs
  constexpr int kRingConsumers = 2 + 2 * kEpiWarps + (kFused ? 2 * (kDecThreads / 32) : 0);

  // stage layout: KS A tiles, KS B_hi halves, KS B_lo halves, then the packed rows
  constexpr int KS = C::KS;
  static_assert(KS == 1 || !kFused, "decoding here loads one K block per stage");
  auto sA = [&](int s, int h) { return base + s * C::kStageBytes + h * A_BYTES; };
  auto sBhi = [&](int s, int h) { return base + s * C::kStageBytes + KS * A_BYTES + h * HB_BYTES; };
  auto sBlo = [&](int s, int h) {
    return base + s * C::kStageBytes + KS * (A_BYTES + HB_BYTES) + h * HB_BYTES;
  };
  auto sPk = [&](int s) { return base + s * C::kStageBytes + KS * (A_BYTES + 2 * HB_BYTES); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t peer_abort = map_to_rank(smem_u32((const void*)abort_flag), rank ^ 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      // the leader's full barrier: its own arrive.expect_tx, plus one arrival per decoder warp
      // of both CTAs when the A tiles are decoded here
      mbar_init(full_bar(s), kFused ? 1 + 2 * (kDecThreads / 32) : 1);
      mbar_init(empty_bar(s), 1);
      mbar_init(pfull_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(cfull_bar(a), 1);
      mbar_init(cempty_bar(a), 2 * kEpiWarps);
    }
    for (int r = 0; r < kTileRing; ++r) {
      mbar_init(tfull_bar(r), 1);
      mbar_init(tempty_bar(r), kRingConsumers);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncwarp();
  cluster_sync_all();  // both CTAs' barriers initialised, both TMEM allocations done
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  const int n_mp = (n_mt + 1) / 2;
  const int num_tiles = n_mp * n_nt;
  const int ckb = chunk_kb(ep);
  const int cid = (int)cluster_id(), ncl = (int)num_clusters();
  // a timeout in either CTA stops both
  auto wait = [&](uint32_t bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, abort_flag, spin_ns, ep.status);
    if (!ok) st_cluster_u32(peer_abort, 1u);
    return ok;
  };
  // Tile `i` of this pair's sequence from the ring, for every consumer role: a single thread
  // (whole_warp false) or a whole warp, whose lane 0 then arrives for it. Returns num_tiles at
  // the end of the work, and -1 on timeout or abort.
  auto take_tile = [&](int i, bool whole_warp) -> int {
    const int r = i % kTileRing;
    if (!mbar_wait_cluster(tfull_bar(r), (uint32_t)(i / kTileRing) & 1u, abort_flag, spin_ns,
                           ep.status)) {
      st_cluster_u32(peer_abort, 1u);
      return -1;
    }
    const int t = tile_slot[r];
    if (whole_warp) __syncwarp();
    if (!whole_warp || lane == 0) mbar_arrive_cluster(map_to_rank(tempty_bar(r), 0u));
    return t;
  };

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kLow));
    if (warp == 0 && lane == 0) {
      // ---------------------------------------------------------- TMA producer (both CTAs)
      int stage = 0;
      uint32_t phase = 0;
      int armed[S];
#pragma unroll
      for (int s = 0; s < S; ++s) armed[s] = -1;
      bool ok = true;
      for (int i = 0; ok; ++i) {
        int tile;
        if (leader) {  // take the next tile and publish it to both CTAs
          const int r = i % kTileRing;
          if (!mbar_wait_cluster(tempty_bar(r), ((uint32_t)(i / kTileRing) & 1u) ^ 1u, abort_flag,
                                 spin_ns, ep.status)) {
            st_cluster_u32(peer_abort, 1u);
            break;
          }
          tile = next_tile(ep.wave_ctr, i, cid, ncl, num_tiles);
          tile_slot[r] = tile;
          st_cluster_u32(map_to_rank(smem_u32((const void*)(tile_slot + r)), 1u), (uint32_t)tile);
          mbar_arrive(tfull_bar(r));
          mbar_arrive_cluster(map_to_rank(tfull_bar(r), 1u));
        } else {
          tile = take_tile(i, false);
          if (tile < 0) break;
        }
        if (tile >= num_tiles) break;
        int mp, nt;
        tile_coord2(tile, n_mp, n_nt, group_p, mp, nt);
        const bool rev = k_reversed(tile, ncl);
        const int mt0 = 2 * mp;
        const uint32_t pair_bytes = 2u * KS * ((kFused ? 0u : (uint32_t)A_BYTES) + 2 * HB_BYTES);
        const int arow = (mt0 + (int)rank) * TBM;
        const int brow = nt * TBN + (int)rank * 128;
        for (int kb = 0; kb < num_kb; kb += KS) {
          const int kx = rev ? num_kb - KS - kb : kb;  // first K block of this stage
          if (!wait(empty_bar(stage), phase ^ 1u)) {
            ok = false;
            break;
          }
          if (*abort_flag) {
            ok = false;
            break;
          }
          if (leader) mbar_expect_tx(full_bar(stage), pair_bytes);
          armed[stage] = (int)phase;
          const uint32_t fb = map_to_rank(full_bar(stage), 0u);
          if (kFused) {  // this CTA's packed rows, completing on its own barrier
            mbar_expect_tx(pfull_bar(stage), (uint32_t)DecCfg<OPA>::kPackBytes);
            tma_load_2d(&da.tmG, sPk(stage), pfull_bar(stage), dec_box_x<OPA>(kx), arow);
          }
#pragma unroll
          for (int h = 0; h < KS; ++h) {
            if (!kFused) tma_load_2d_pair(&tmAhi, sA(stage, h), fb, (kx + h) * TBK, arow);
            tma_load_2d_pair(&tmBhi, sBhi(stage, h), fb, (kx + h) * TBK, brow);
            tma_load_2d_pair(&tmBlo, sBlo(stage, h), fb, (kx + h) * TBK, brow);
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // the leader's armed stages complete only when both CTAs' copies have landed; the packed
      // rows of every CTA land in its own barrier (bounded)
      for (int s = 0; s < S; ++s) {
        if (armed[s] < 0) continue;
        if (kFused) mbar_wait(pfull_bar(s), (uint32_t)armed[s], abort_flag, spin_ns, ep.status);
        if (leader) mbar_wait(full_bar(s), (uint32_t)armed[s], abort_flag, spin_ns, ep.status);
      }
    } else if (warp == 1 && lane == 0 && leader) {
      // ---------------------------------------------------------- MMA issuer (leader)
      int stage = 0;
      uint32_t phase = 0;
      uint32_t g = 0;
      bool ok = true;
      for (int i = 0; ok; ++i) {
        const int tile = take_tile(i, false);
        if (tile < 0 || tile >= num_tiles) break;
        for (int kb0 = 0; kb0 < num_kb && ok; kb0 = chunk_end_c(kb0, num_kb, ckb), ++g) {
          const int acc = (int)(g & 1u);
          const uint32_t ph = (g >> 1) & 1u;
          if (!wait(cempty_bar(acc), ph ^ 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(acc * TBN);
          const int kb1 = chunk_end_c(kb0, num_kb, ckb);
          for (int kb = kb0; kb < kb1; kb += KS) {
            if (!wait(full_bar(stage), phase)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < KS; ++h)
#pragma unroll
              for (int k = 0; k < TBK / 16; ++k) {
                const uint64_t a = sdesc_sw64(sA(stage, h) + 32u * k);
                const uint64_t bh = sdesc_sw64(sBhi(stage, h) + 32u * k);
                const uint64_t bl = sdesc_sw64(sBlo(stage, h) + 32u * k);
                tc2_mma(d, a, bh, (kb > kb0 || h > 0 || k > 0) ? 1u : 0u);
                tc2_mma(d, a, bl, 1u);
              }
            tc2_commit_both(empty_bar(stage));
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (ok) tc2_commit_both(cfull_bar(acc));
        }
      }
      tc2_commit_local(drain_bar);
      mbar_wait(drain_bar, 0u, abort_flag, spin_ns, ep.status);
    } else if (kFused && warp >= 2) {
      // ---------------------------------------------------------- decoders (both CTAs)
      const int t = threadIdx.x - 64;  // rows t and t + 64 of this CTA's A tile
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int i = 0; ok; ++i) {
        const int tile = take_tile(i, true);
        if (tile < 0 || tile >= num_tiles) break;
        int mp, nt;
        tile_coord2(tile, n_mp, n_nt, group_p, mp, nt);
        const long long r0 = (long long)(2 * mp + (int)rank) * TBM + t;
        const uint2 k0 = dec_row_consts<OPA>(da, r0), k1 = dec_row_consts<OPA>(da, r0 + 64);
        const bool rev = k_reversed(tile, ncl);
        for (int kb = 0; kb < num_kb; ++kb) {
          const int kx = rev ? num_kb - 1 - kb : kb;  // the K block the producer loaded
          if (!wait(pfull_bar(stage), phase)) {
            ok = false;
            break;
          }
          dec_expand_store<OPA>(sPk(stage), k0, r0 < da.M, t, kx, da.N, sA(stage, 0));
          dec_expand_store<OPA>(sPk(stage), k1, r0 + 64 < da.M, t + 64, kx, da.N, sA(stage, 0));
          // the leader's tensor core reads this CTA's tile: make the stores visible to the
          // async proxy at cluster scope before signalling
          asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(map_to_rank(full_bar(stage), 0u));
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kHigh));
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;
    const uint32_t leader_cempty0 = map_to_rank(cempty_bar(0), 0u);
    const uint32_t leader_cempty1 = map_to_rank(cempty_bar(1), 0u);
    uint32_t g = 0;
    bool ok = true;
    for (int i = 0; ok; ++i) {
      const int tile = take_tile(i, true);
      if (tile < 0 || tile >= num_tiles) break;
      int mp, nt;
      tile_coord2(tile, n_mp, n_nt, group_p, mp, nt);
      float tot[128];
#pragma unroll
      for (int e = 0; e < 128; ++e) tot[e] = 0.0f;
      for (int kb0 = 0; kb0 < num_kb; kb0 = chunk_end_c(kb0, num_kb, ckb), ++g) {
        const int acc = (int)(g & 1u);
        const uint32_t ph = (g >> 1) & 1u;
        if (!wait(cfull_bar(acc), ph)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(acc * TBN + half * 128);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float v[32];
          __syncwarp();  // tcgen05.ld is .sync.aligned
          tc_ld32(taddr + (uint32_t)(i * 32), v);
#pragma unroll
          for (int e = 0; e < 32; ++e) tot[i * 32 + e] += v[e];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(acc ? leader_cempty1 : leader_cempty0);
      }
      if (!ok) break;
      const long long row_base = (long long)(2 * mp + (int)rank) * TBM + quarter * 32;
      const long long row = row_base + lane;
      const bool row_ok = row < ep.M;
      const float rinv = row_ok ? ep.row_inv[row] : __int_as_float(0x7fc00000);
      const float shift = (row_ok && ep.row_shift) ? ep.row_shift[row] : 0.0f;
      epilogue_tile(ep, tot, row, row_base, row_ok, rinv, shift, nt * TBN + half * 128, lane);
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  cluster_sync_all();  // neither CTA leaves while the other may still signal its barriers
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

template <int OPA>
cudaError_t go2(const CUtensorMap* a, const CUtensorMap* bh, const CUtensorMap* bl, int64_t K,
                const EpiParams& ep, int sm_count, int group_m, long long spin_ns, cudaStream_t st,
                const DecodeArgs& da) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc2_scan<OPA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg2<OPA>::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + TBM - 1) / TBM;
  const int n_nt = (ep.P + TBN - 1) / TBN;
  const int tiles = ((n_mt + 1) / 2) * n_nt;
  const int pairs = tiles < sm_count / 2 ? tiles : sm_count / 2;
  const int group_p = group_m / 2 > 0 ? group_m / 2 : 1;
  if ((K / TBK) % Cfg2<OPA>::KS) return cudaErrorInvalidValue;
  k_tc2_scan<OPA><<<2 * pairs, kThreads, Cfg2<OPA>::kSmem, st>>>(
      *a, *bh, *bl, (int)(K / TBK), n_mt, n_nt, group_p, spin_ns, ep, da);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc2_scan(const CUtensorMap* tmA, const CUtensorMap* tmBhi,
                            const CUtensorMap* tmBlo, int64_t K, const EpiParams& ep, int sm_count,
                            long long spin_ns, cudaStream_t st, int group_m, const DecodeArgs* dec,
                            int encoding) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  if (K % TBK || group_m < 1) return cudaErrorInvalidValue;
  if (!dec)
    return go2<OPA_TMA>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, DecodeArgs{});
  if (dec->M != ep.M) return cudaErrorInvalidValue;
  if (encoding == TG_ENC_2BIT)
    return go2<OPA_2BIT>(tmBhi, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, *dec);
  return go2<OPA_U8>(tmBhi, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, *dec);
}

}  // namespace tg
