// Tensor-core scan: Eq. 2 of Section 2.2 on tcgen05, fused with Eq. 3 and the p-value.
//
// D = A (B_hi + B_lo)^T + c (sum_i B) for a block of markers against the whole panel:
//   A     [M][K] bf16  each marker row shifted by its c (exact), bf16(mean - c) at a missing call
//   B_hi, B_lo [P][K]  bf16 split of the unit-norm residualised panel, y ~= hi + lo
//   c (per row), sum_i B (per column) added back in the epilogue
// K = samples (zero padded), FP32 accumulation in tensor memory.
//
// Persistent kernel, one CTA per SM, 384 threads (3 warpgroups), warp-specialised:
//   warp 0 lane 0  TMA producer: 128x32 A tiles and 256x32 B tiles (64-byte swizzle) into a
//                  ring of shared-memory stages, completion tracked by mbarrier transaction bytes
//   warps 2, 3     with packed genotypes instead of a decoded operand (OPA_2BIT / OPA_U8): the
//                  decoders, which expand each A tile from the packed rows (tc_common.cuh) and
//                  join the stage's full barrier
//   warp 1 lane 0  MMA issuer: per 32-wide K step, 2 x 2 tcgen05.mma 128x256x16 into an
//                  FP32 accumulator in TMEM
//   warps 4..11    epilogue: tcgen05.ld of the accumulator (thread = marker row, each warp one
//                  TMEM lane quarter and one half of the 256 columns), r = D / |g_res|, hits
//                  above the r^2 threshold, per-phenotype best marker, optionally every statistic.
// Accumulation is chunked: the tensor core sums at most 1024 samples (32 K blocks) into a
// fresh TMEM accumulator, and the epilogue warps add the chunk results into FP32 totals held
// in registers with round-to-nearest adds. The tensor core's FP32 accumulation drops low bits
// toward zero at each chained addition, which over 23,000 samples biases |r| low by about
// 5e-5 relative; chunks of 1024 keep that bias near 2e-6. Two chunk accumulators (512 TMEM
// columns) alternate, so draining one overlaps the products of the next.
// Tiles are 128 x 256, or 128 x 64 for panels of at most 64 phenotypes. 64- and 128-column
// tiles of blocks with at least one 256-marker tile per SM take 256 markers, as two 128-row
// sub-tiles with their own accumulators sharing each B stage (half the B traffic from L2).
// In raw mode (the covariate projection, alone or joint with a small panel whose phenotypes
// follow the q - 1 projection columns in one B operand) the tile is the narrowest of 64, 128
// and 256 columns that holds them, and the products are written unnormalised; k_raw_stats
// turns a joint pass's panel columns into statistics once the marker norms exist.
// With split-K (ep.ksplit > 1, for blocks with fewer tiles than SMs) a work item is a tile and
// a chunk-aligned range of the samples; the tile's first range adds the other ranges' partial
// sums (handed over in global memory) in range order before its epilogue.
// Every wait is bounded: past the limit the kernel latches ST_TIMEOUT, raises a shared abort
// flag, lets in-flight copies and products finish (again bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace tg {
namespace {

using namespace tcx;

template <int OPA, int KS = 1, int BR = 64, int MS = 1>
struct Cfg {
  // A, B_hi, B_lo and (when decoding here) the CTA's packed rows: 40 KB (+ 2 or 4 KB), 5 stages.
  // Two K blocks of MS A sub-tiles and BR B rows: the same slot for MS = 1 and BR = 64, else
  // 2 x (MS x 8 + 2 x BR x 64 B): 48 KB in 4 stages or 64 KB in 3
  static constexpr bool kWide = KS == 2 && (BR > 64 || MS > 1);
  static constexpr int kStageBytes = kWide ? KS * (MS * A_BYTES + 2 * BR * TBK * 2)
                                           : A_BYTES + 2 * B_BYTES + DecCfg<OPA>::kPackBytes;
  static constexpr int kStages = !kWide ? 5 : kStageBytes <= 48 * 1024 ? 4 : 3;
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStageBytes + kBarBytes + 1024;  // + alignment slack
};

// MS = 128-marker sub-tiles per tile (KS = 2 only): with MS = 2 a CTA takes 256 markers, two
// accumulators of 128 TMEM lanes at columns +0 and +128 sharing every B stage, which halves the
// B operand's traffic from L2 into shared memory; each element's products and additions are
// the same as with MS = 1, so the results are too.
// KS = K blocks per stage, BR = B rows per K block when KS = 2. With 64- or 128-column tiles (the
// covariate projection, alone or joint with a small panel, and panels of at most 64 phenotypes)
// the kernel streams the 3 GB operand and is bound by HBM, where two consecutive 64-byte row
// segments requested back to back use the DRAM pages better than one: it then loads two K
// blocks per stage (A halves at 0 and 8 KB, then the two B_hi halves, then the two B_lo halves,
// BR x 64 B each).
static_assert(kChunkKB == kAccumChunkKB, "the host's split choice counts the same chunks");

// K-block range [lo, hi) of split `sp` of `ks`: whole accumulation chunks, the earlier splits
// one chunk longer when they do not divide evenly (a split may be empty).
__device__ __forceinline__ void split_range(int num_kb, int ks, int sp, int& lo, int& hi) {
  const int chunks = (num_kb + kChunkKB - 1) / kChunkKB;
  const int per = (chunks + ks - 1) / ks;
  lo = min(num_kb, sp * per * kChunkKB);
  hi = min(num_kb, (sp + 1) * per * kChunkKB);
}
// End of the accumulation chunk that starts at kb0 within [lo, hi); chunk_end for a whole range.
__device__ __forceinline__ int chunk_end_in(int kb0, int lo, int hi) {
  const int e = kb0 == lo ? lo + kFirstChunks * kChunkKB : kb0 + kChunkKB;
  return e < hi ? e : hi;
}

template <int OPA, int KS, int BR, int MS>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_scan(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmBhi,
              const __grid_constant__ CUtensorMap tmBlo, int num_kb, int n_mt, int n_nt, int bn,
              int group_m, long long spin_ns, EpiParams ep,
              const __grid_constant__ DecodeArgs da) {
  // bn = B rows per tile: 256 for the phenotype panel, 64 or 128 (<= BR) with KS = 2
  using C = Cfg<OPA, KS, BR, MS>;
  static_assert(MS == 1 || (MS == 2 && KS == 2 && BR <= 128), "two sub-tiles: two K blocks, <= 128 B rows");
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
  auto pfull_bar = [&](int s) { return bars + 8u * (2 * S + 5 + s); };  // packed rows landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * C::kStageBytes + 8 * (3 * S + 5));
  static_assert(8 * (3 * S + 5) + 8 <= C::kBarBytes, "barrier area");
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  auto sA = [&](int s) { return base + s * C::kStageBytes; };
  auto sBhi = [&](int s) { return base + s * C::kStageBytes + A_BYTES; };
  auto sBlo = [&](int s) { return base + s * C::kStageBytes + A_BYTES + B_BYTES; };
  auto sPk = [&](int s) { return base + s * C::kStageBytes + A_BYTES + 2 * B_BYTES; };
  constexpr int kBk = BR * TBK * 2;   // one K block of B rows (KS = 2)
  constexpr int kAk = MS * A_BYTES;   // one K block of A rows (KS = 2)
  static_assert(KS == 1 || (KS == 2 && !kFused && 2 * kAk + 4 * kBk <= C::kStageBytes),
                "two K blocks per stage: decoded operand and at most BR B rows");
  auto sAk = [&](int s, int h, int sub) {
    return KS == 1 ? sA(s) : sA(s) + (uint32_t)(h * kAk + sub * A_BYTES);
  };
  auto sBhik = [&](int s, int h) {
    return KS == 1 ? sBhi(s) : sA(s) + (uint32_t)(2 * kAk + h * kBk);
  };
  auto sBlok = [&](int s, int h) {
    return KS == 1 ? sBlo(s) : sA(s) + (uint32_t)(2 * kAk + 2 * kBk + h * kBk);
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), kFused ? 1 + kDecThreads / 32 : 1);  // + one arrival per decoder warp
      mbar_init(empty_bar(s), 1);
      mbar_init(pfull_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(cfull_bar(a), 1);
      mbar_init(cempty_bar(a), kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  const int num_tiles = n_mt * n_nt;
  // work items: (tile, split); a tile's ks items are consecutive and run in the same round
  // (the grid is a multiple of ks and every CTA is resident)
  const int ks = ep.ksplit > 1 ? ep.ksplit : 1;
  const int num_items = num_tiles * ks;
  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kLow));
    if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int stage = 0;
    uint32_t phase = 0;
    int armed[S];
#pragma unroll
    for (int s = 0; s < S; ++s) armed[s] = -1;
    bool ok = true;
    for (int item = blockIdx.x; item < num_items && ok; item += gridDim.x) {
      const int tile = item / ks;
      int mt, nt, kb_lo, kb_hi;
      tile_coord(tile, n_mt, n_nt, group_m, mt, nt);
      split_range(num_kb, ks, item - tile * ks, kb_lo, kb_hi);
      const uint32_t bytes =
          (uint32_t)KS * ((kFused ? 0u : (uint32_t)kAk) + 2u * (uint32_t)bn * (TBK * 2));
      for (int kb = kb_lo; kb < kb_hi; kb += KS) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full_bar(stage), bytes);
        armed[stage] = (int)phase;
        if (kFused) {
          mbar_expect_tx(pfull_bar(stage), (uint32_t)DecCfg<OPA>::kPackBytes);
          tma_load_2d(&da.tmG, sPk(stage), pfull_bar(stage), dec_box_x<OPA>(kb), mt * TBM);
        }
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          if (!kFused)
#pragma unroll
            for (int sub = 0; sub < MS; ++sub)
              tma_load_2d(&tmAhi, sAk(stage, h, sub), full_bar(stage), (kb + h) * TBK,
                          (mt * MS + sub) * TBM);
          tma_load_2d(&tmBhi, sBhik(stage, h), full_bar(stage), (kb + h) * TBK, nt * bn);
          tma_load_2d(&tmBlo, sBlok(stage, h), full_bar(stage), (kb + h) * TBK, nt * bn);
        }
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // copies still in flight land before the CTA leaves (bounded)
    for (int s = 0; s < S; ++s)
      if (armed[s] >= 0) {
        if (kFused) mbar_wait(pfull_bar(s), (uint32_t)armed[s], abort_flag, spin_ns, ep.status);
        mbar_wait(full_bar(s), (uint32_t)armed[s], abort_flag, spin_ns, ep.status);
      }
    } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    // Each chunk (chunk_end) starts a fresh accumulator (no chained accumulation
    // across chunks); the two chunk accumulators alternate.
    int stage = 0;
    uint32_t phase = 0;
    uint32_t g = 0;
    bool ok = true;
    const uint32_t idesc = idesc_bf16(bn);
    for (int item = blockIdx.x; item < num_items && ok; item += gridDim.x) {
      const int tile = item / ks;
      int kb_lo, kb_hi;
      split_range(num_kb, ks, item - tile * ks, kb_lo, kb_hi);
      for (int kb0 = kb_lo; kb0 < kb_hi && ok; kb0 = chunk_end_in(kb0, kb_lo, kb_hi), ++g) {
        const int acc = (int)(g & 1u);
        const uint32_t ph = (g >> 1) & 1u;
        if (!mbar_wait(cempty_bar(acc), ph ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * TBN);
        const int kb1 = chunk_end_in(kb0, kb_lo, kb_hi);
        for (int kb = kb0; kb < kb1; kb += KS) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, spin_ns, ep.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int h = 0; h < KS; ++h)
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k) {
              const uint64_t bh = sdesc_sw64(sBhik(stage, h) + 32u * k);
              const uint64_t bl = sdesc_sw64(sBlok(stage, h) + 32u * k);
#pragma unroll
              for (int sub = 0; sub < MS; ++sub) {  // sub-tile accumulators at +0 and +128
                const uint64_t a = sdesc_sw64(sAk(stage, h, sub) + 32u * k);
                const uint32_t ds = d + (uint32_t)(sub * 128);
                tc_mma(ds, a, bh, idesc, (kb > kb0 || h > 0 || k > 0) ? 1u : 0u);
                tc_mma(ds, a, bl, idesc, 1u);
              }
            }
          tc_commit(empty_bar(stage));
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) tc_commit(cfull_bar(acc));
      }
    }
    // every product issued so far completes before TMEM is released (bounded)
    tc_commit(drain_bar);
    mbar_wait(drain_bar, 0u, abort_flag, spin_ns, ep.status);
    } else if (kFused && warp >= 2) {
    // ------------------------------------------------------------ decoders (warps 2, 3)
    const int t = threadIdx.x - 64;  // rows t and t + 64 of each A tile
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < num_items && ok; item += gridDim.x) {
      const int tile = item / ks;
      int mt, nt, kb_lo, kb_hi;
      tile_coord(tile, n_mt, n_nt, group_m, mt, nt);
      split_range(num_kb, ks, item - tile * ks, kb_lo, kb_hi);
      const long long r0 = (long long)mt * TBM + t;
      const uint2 k0 = dec_row_consts<OPA>(da, r0), k1 = dec_row_consts<OPA>(da, r0 + 64);
      for (int kb = kb_lo; kb < kb_hi; ++kb) {
        if (!mbar_wait(pfull_bar(stage), phase, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        dec_expand_store<OPA>(sPk(stage), k0, r0 < da.M, t, kb, da.N, sA(stage));
        dec_expand_store<OPA>(sPk(stage), k1, r0 + 64 < da.M, t + 64, kb, da.N, sA(stage));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
        __syncwarp();
        if (lane == 0) mbar_arrive(full_bar(stage));
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kHigh));
    // ------------------------------------------------------------ epilogue
    // 8 warps: (TMEM lane quarter, column half) pairs; FP32 running totals in registers.
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;
    uint32_t g = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < num_items && ok; item += gridDim.x) {
      const int tile = item / ks, split = item - tile * ks;
      int mt, nt, kb_lo, kb_hi;
      tile_coord(tile, n_mt, n_nt, group_m, mt, nt);
      split_range(num_kb, ks, split, kb_lo, kb_hi);
      float tot[128];
#pragma unroll
      for (int e = 0; e < 128; ++e) tot[e] = 0.0f;
      for (int kb0 = kb_lo; kb0 < kb_hi; kb0 = chunk_end_in(kb0, kb_lo, kb_hi), ++g) {
        const int acc = (int)(g & 1u);
        const uint32_t ph = (g >> 1) & 1u;
        if (!mbar_wait(cfull_bar(acc), ph, abort_flag, spin_ns, ep.status)) {
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
        if (lane == 0) mbar_arrive(cempty_bar(acc));
      }
      if (!ok) break;
      if (ks > 1) {
        // this thread's row and 128 columns of the tile's partial sums
        const int rc = (quarter * 32 + lane) * TBN + half * 128;
        float* wsp = ep.sk_ws + (size_t)tile * (size_t)(ks - 1) * (TBM * TBN);
        if (split > 0) {  // hand the partial sums to the tile's split 0, warp by warp
          float4* dst = reinterpret_cast<float4*>(wsp + (size_t)(split - 1) * (TBM * TBN) + rc);
#pragma unroll
          for (int e = 0; e < 32; ++e)
            dst[e] = make_float4(tot[4 * e], tot[4 * e + 1], tot[4 * e + 2], tot[4 * e + 3]);
          __threadfence();
          __syncwarp();
          if (lane == 0) atomicAdd(ep.sk_cnt + tile, 1u);
          continue;
        }
        // split 0: each warp waits (bounded) for the other splits' warps, then adds their sums
        // in split order; no CTA-wide barrier, so a warp that gave up cannot hold the others
        bool got = true;
        if (lane == 0) {
          const unsigned need = (unsigned)((ks - 1) * kEpiWarps);
          const uint64_t t0 = globaltimer_ns();
          while (*reinterpret_cast<volatile unsigned*>(ep.sk_cnt + tile) < need) {
            if (*abort_flag || (long long)(globaltimer_ns() - t0) > spin_ns) {
              if (!*abort_flag) {
                *abort_flag = 1;
                atomicOr(ep.status, ST_TIMEOUT);
              }
              got = false;
              break;
            }
            __nanosleep(128);
          }
          __threadfence();
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();  // the partial sums are read after lane 0 saw them complete
        if (!got) {
          ok = false;
          break;
        }
        for (int sp = 1; sp < ks; ++sp) {
          const float4* src =
              reinterpret_cast<const float4*>(wsp + (size_t)(sp - 1) * (TBM * TBN) + rc);
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const float4 v = __ldcg(src + e);
            tot[4 * e] += v.x;
            tot[4 * e + 1] += v.y;
            tot[4 * e + 2] += v.z;
            tot[4 * e + 3] += v.w;
          }
        }
      }
      // MS = 1: warps of half h hold columns h*128.. of the tile's 128 rows; MS = 2: warps of
      // half h hold the (at most 128) columns of sub-tile h's 128 rows
      const long long row_base =
          (long long)(MS == 2 ? (mt * MS + half) : mt) * TBM + quarter * 32;
      const int col_half = MS == 2 ? 0 : half * 128;
      const long long row = row_base + lane;
      const bool row_ok = row < ep.M;
      const float rinv = (row_ok && ep.row_inv) ? ep.row_inv[row] : __int_as_float(0x7fc00000);
      const float shift = (row_ok && ep.row_shift) ? ep.row_shift[row] : 0.0f;
      if (ep.raw_out) {
        // covariate projection (and a small panel's products): the first raw_cols columns of
        // the tile, unnormalised
        if (row_ok) {
#pragma unroll
          for (int e = 0; e < 128; ++e) {  // fully unrolled: tot stays in registers
            const int col = col_half + e;
            if (col < ep.raw_cols)
              ep.raw_out[row * ep.raw_ld + col] = fmaf(shift, ep.col_cs[col], tot[e]);
          }
        }
      } else {
        epilogue_tile(ep, tot, row, row_base, row_ok, rinv, shift,
                      (MS == 2 ? nt * bn : nt * TBN) + col_half, lane);
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// Statistics of a small panel from its raw products: a block takes 64 consecutive marker rows,
// its threads split into 256 / P groups of P (thread = phenotype column) that take every
// (256 / P)-th row, so each row is read coalesced and a small panel still keeps the block busy.
// Per element the arithmetic of the contraction epilogue (D already holds the shift's add-back):
// r = D / |a_res| clamped, the hit test on r^2, r in FULL mode, and the key (|r| bits, ~marker)
// whose maximum is the column's best marker; the groups' keys meet in shared memory and each
// column offers one per block.
constexpr int kRawRows = 64;
constexpr int kRawThreads = 256;
static_assert(JCOLS <= kRawThreads, "a group of P threads per block");
__global__ void __launch_bounds__(kRawThreads) k_raw_stats(const float* __restrict__ raw,
                                                           long long ld, EpiParams ep) {
  __shared__ unsigned long long keys[kRawThreads];
  __shared__ int has[kRawThreads];
  const int groups = kRawThreads / ep.P;  // P <= JCOLS <= kRawThreads
  const int col = (int)threadIdx.x % ep.P, sub = (int)threadIdx.x / ep.P;
  const bool active = sub < groups;
  const long long r0 = (long long)blockIdx.x * kRawRows;
  const long long r1 = r0 + kRawRows < (long long)ep.M ? r0 + kRawRows : (long long)ep.M;
  unsigned long long best = 0;
  bool any = false;
  if (active) {
    const float rmul = ep.col_rmul[col];
    for (long long row = r0 + sub; row < r1; row += groups) {
      const float D = raw[row * ld + col];
      const float r = corr_nan(D, ep.row_inv[row], rmul);
      if (ep.do_hits && r * r >= ep.r2_thr) emit_hit_raw(ep, D, row, col);
      if (ep.do_full) ep.rstore[row * ep.ldo + col] = r;
      if (r == r) {
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(fabsf(r)) << 32) |
            (unsigned long long)(0xFFFFFFFFu - (uint32_t)(ep.marker_offset + row));
        best = key > best ? key : best;
        any = true;
      }
    }
  }
  if (!ep.do_best) return;  // the same for every thread of the launch
  keys[threadIdx.x] = best;
  has[threadIdx.x] = any ? 1 : 0;
  __syncthreads();
  if (active && sub == 0) {
    for (int g = 1; g < groups; ++g) {
      const int t = g * ep.P + col;
      if (has[t]) {
        best = keys[t] > best ? keys[t] : best;
        any = true;
      }
    }
    if (any) best_offer(ep.best + col, best);
  }
}

__global__ void k_wait_test(const volatile uint32_t* flag, long long limit_ns, uint32_t* result) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (*flag) {
      *result = 1u;
      return;
    }
    if ((long long)(globaltimer_ns() - t0) > limit_ns) {
      *result = 2u;
      return;
    }
    __nanosleep(1000);
  }
}

template <int OPA, int KS, int BR = 64, int MS = 1>
cudaError_t go(const CUtensorMap* a, const CUtensorMap* bh, const CUtensorMap* bl, int64_t K,
               const EpiParams& ep, int sm_count, int group_m, long long spin_ns, cudaStream_t st,
               const DecodeArgs& da, int bn) {
  static bool attr_set = false;  // per process and instantiation; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_scan<OPA, KS, BR, MS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg<OPA, KS, BR, MS>::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + MS * TBM - 1) / (MS * TBM);
  const int n_nt = (ep.P + bn - 1) / bn;
  const int ks = ep.ksplit > 1 ? ep.ksplit : 1;
  if (ks > 1 && (!ep.sk_ws || !ep.sk_cnt || sm_count < ks))
    return cudaErrorInvalidValue;
  const int items = n_mt * n_nt * ks;
  // a multiple of ks, so that the splits of a tile run in the same round
  const int grid = (items < sm_count ? items : sm_count) / ks * ks;
  if (KS == 2 && (bn > BR || (K / TBK) % 2)) return cudaErrorInvalidValue;
  k_tc_scan<OPA, KS, BR, MS><<<grid, kThreads, Cfg<OPA, KS, BR, MS>::kSmem, st>>>(
      *a, *bh, *bl, (int)(K / TBK), n_mt, n_nt, bn, group_m, spin_ns, ep, da);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_scan(const CUtensorMap* tmA, const CUtensorMap* tmBhi,
                           const CUtensorMap* tmBlo, int64_t K, const EpiParams& ep, int sm_count,
                           long long spin_ns, cudaStream_t st, int group_m, const DecodeArgs* dec,
                           int encoding, bool narrow) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  if (K % TBK || group_m < 1) return cudaErrorInvalidValue;
  // raw mode: the narrowest tile that holds the raw columns (the B maps' boxes match)
  const int bn = narrow ? 64
                 : ep.raw_out ? (ep.raw_cols <= 64 ? 64 : ep.raw_cols <= 128 ? 128 : TBN)
                              : TBN;
  if (narrow && ep.P > 64) return cudaErrorInvalidValue;
  if (ep.raw_out && (ep.raw_cols > TBN || ep.P != ep.raw_cols)) return cudaErrorInvalidValue;
  if (!dec) {
    // 256-marker tiles (two sub-tiles sharing B) once they fill every SM at least once, and
    // not with split-K, whose workspace the host sized for 128-marker tiles
    const bool two = ep.ksplit <= 1 && (ep.M + 2 * TBM - 1) / (2 * TBM) >= sm_count;
    if (bn == 64)  // the covariate projection, or a panel of at most 64 phenotypes
      return two ? go<OPA_TMA, 2, 64, 2>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns,
                                         st, DecodeArgs{}, bn)
                 : go<OPA_TMA, 2, 64, 1>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns,
                                         st, DecodeArgs{}, bn);
    if (bn == 128)  // the projection joint with a panel of at most 128 - (q - 1) phenotypes
      return two ? go<OPA_TMA, 2, 128, 2>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns,
                                          st, DecodeArgs{}, bn)
                 : go<OPA_TMA, 2, 128, 1>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns,
                                          st, DecodeArgs{}, bn);
    return go<OPA_TMA, 1>(tmA, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, DecodeArgs{},
                          bn);
  }
  if (dec->M != ep.M) return cudaErrorInvalidValue;
  if (encoding == TG_ENC_2BIT)
    return go<OPA_2BIT, 1>(tmBhi, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, *dec, bn);
  return go<OPA_U8, 1>(tmBhi, tmBhi, tmBlo, K, ep, sm_count, group_m, spin_ns, st, *dec, bn);
}

cudaError_t launch_raw_stats(const float* raw, int64_t ld, const EpiParams& ep, cudaStream_t st) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  if (ep.P > JCOLS) return cudaErrorInvalidValue;
  const long long blocks = ((long long)ep.M + kRawRows - 1) / kRawRows;
  k_raw_stats<<<(unsigned)blocks, kRawThreads, 0, st>>>(raw, (long long)ld, ep);
  return cudaGetLastError();
}

cudaError_t launch_wait_test(const uint32_t* flag, long long limit_ns, uint32_t* result,
                             cudaStream_t st) {
  k_wait_test<<<1, 1, 0, st>>>(flag, limit_ns, result);
  return cudaGetLastError();
}

}  // namespace tg
