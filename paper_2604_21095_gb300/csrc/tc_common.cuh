// Pieces shared by the two tcgen05 scan kernels (one CTA per tile, and CTA pairs):
// tile constants, PTX wrappers for mbarriers, TMA, tcgen05 fences and TMEM loads, the bounded
// wait, and the statistics epilogue of one thread's 128 running totals.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "genotype.cuh"
#include "internal.h"

namespace tg {
namespace tcx {

constexpr int TBM = 128, TBN = 256, TBK = 32;  // TBK bf16 = 64 bytes = one swizzle row
constexpr int A_BYTES = TBM * TBK * 2;         // 8 KB
constexpr int B_BYTES = TBN * TBK * 2;         // 16 KB
constexpr int kEpiWarps = 8;
// Three warpgroups: warpgroup 0 = producer warp, MMA warp and two decoder warps (idle when the
// A operand comes by TMA); warpgroups 1-2 = the 8 epilogue warps. At launch every thread gets 168 registers (384 x 168 = 64,512); then
// warpgroup 0 gives registers back (56 each) and the epilogue warpgroups take them
// (224 each): 128 x 56 + 256 x 224 = 64,512, the launch total, so the increase cannot stall.
// When warps 2-3 decode the A operand (see below) they need more: 64 / 216
// (128 x 64 + 256 x 216 = 63,488).
constexpr int kThreads = 384;
template <int OPA>
struct RegSplit {
  static constexpr int kLow = OPA == 0 ? 56 : 64;
  static constexpr int kHigh = OPA == 0 ? 224 : 216;
  static_assert(128 * kLow + 256 * kHigh <= kThreads * 168, "register split exceeds launch");
};
constexpr int kTmemCols = 512;                 // two 128 x 256 FP32 chunk accumulators
constexpr int kChunkKB = 32;                   // K blocks per accumulation chunk (1024 samples)
// The first chunk of each tile is kFirstChunks chunks long: the epilogue warps finish the
// previous tile's statistics while it runs, and a longer first chunk gives them that time
// before the products need a drained accumulator again (one longer chunk in ~20 changes the
// accumulation little).
constexpr int kFirstChunks = 1;
__host__ __device__ constexpr int chunk_end(int kb0, int num_kb) {
  return (kb0 == 0 ? kFirstChunks * kChunkKB : kb0 + kChunkKB) < num_kb
             ? (kb0 == 0 ? kFirstChunks * kChunkKB : kb0 + kChunkKB)
             : num_kb;
}



// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_m(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int n) { return idesc_bf16_m(TBM, n); }
// The same with A = B = F16 (type code 0 in bits 7-9 and 10-12), M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of 64 bytes,
// 8-row core groups 512 bytes apart (SBO), version 1, start address >> 4.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // layout: 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait for the completion of phase `parity`; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       long long limit_ns, uint32_t* status) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((long long)(globaltimer_ns() - t0) > limit_ns) {
      *abort_flag = 1;
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint32_t dst, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ decode in the producer
// Operand kinds of the contraction kernels: A by TMA from a decoded operand in HBM, or decoded
// from packed genotypes (OPA_2BIT, OPA_U8). In the second case the producer thread also loads,
// by TMA, the CTA's 128 packed rows for each K block into the stage (a box of 32 bytes per row
// for dosages, one K block; 16 bytes for 2-bit calls, two K blocks of which the stage uses one
// half), completing on the stage's packed-full barrier; the decoder warps (warps 2 and 3, 64
// threads, two rows each) wait on it, expand the rows to the centred split operand
// (genotype.cuh), store each row's four 16-byte chunks where the TMA's 64-byte swizzle would
// put them (chunk j of row r at r * 64 + 16 * (j ^ ((r >> 1) & 3))) and join the stage's full
// barrier. The packed load is issued after the stage's empty barrier, so a completed
// packed-full barrier also means the A tile may be overwritten.
enum { OPA_TMA = 0, OPA_2BIT = 1, OPA_U8 = 2 };
constexpr int kDecThreads = 64;
template <int OPA>
struct DecCfg {
  static constexpr int kBox = OPA == OPA_U8 ? 32 : 16;  // packed bytes per row in a stage
  static constexpr int kPackBytes = OPA == OPA_TMA ? 0 : TBM * kBox;
};

// Per-row constants of the expansion: 2-bit {lut0, lut1}, dosage {2^23 + c as float bits, mh2}.
template <int OPA>
__device__ __forceinline__ uint2 dec_row_consts(const DecodeArgs& da, long long row) {
  if (row >= da.M) return make_uint2(0u, 0u);
  const float c = da.shift[row];
  const uint32_t mh = da.mh[row] & 0xFFFFu;
  if (OPA == OPA_2BIT)
    return make_uint2(bf16_bits(2.0f - c) | (mh << 16), bf16_bits(1.0f - c) | (bf16_bits(-c) << 16));
  return make_uint2(__float_as_uint(8388608.0f + c), mh | (mh << 16));
}

// Expand row r's K block kb from the stage's packed rows and store it, swizzled, into the A
// tile; one 16-sample half (two 16-byte chunks) at a time.
template <int OPA>
__device__ __forceinline__ void dec_expand_store(uint32_t packed, uint2 k, bool row_ok, int r,
                                                 int kb, int N, uint32_t a_tile) {
  constexpr int BOX = DecCfg<OPA>::kBox;
  const uint32_t src = packed + (uint32_t)(r * BOX) + (OPA == OPA_2BIT ? 8u * (uint32_t)(kb & 1) : 0u);
  const uint32_t row_base = a_tile + (uint32_t)r * 64u;
  const uint32_t sw = (uint32_t)((r >> 1) & 3);
#pragma unroll 1  // rolled: unrolled, the dosage form spilled in the CTA-pair kernel
  for (int h = 0; h < 2; ++h) {
    uint32_t o[8];
    if (OPA == OPA_2BIT) {
      uint32_t w;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w) : "r"(src + 4 * h));
      split16_2bit(w, k.x, k.y, o);
    } else {
      uint4 v;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                   : "r"(src + 16 * h));
      split16_u8(v, __uint_as_float(k.x), 0u, k.y, o);
    }
    const int i0 = kb * TBK + 16 * h;
    if (!row_ok) {
#pragma unroll
      for (int p = 0; p < 8; ++p) o[p] = 0u;
    } else if (i0 + 16 > N) {
      zero_tail16(o, i0, N);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const uint32_t j = (uint32_t)(2 * h + c);
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(row_base + ((j ^ sw) << 4)),
                   "r"(o[4 * c]), "r"(o[4 * c + 1]), "r"(o[4 * c + 2]), "r"(o[4 * c + 3])
                   : "memory");
    }
  }
}

// x coordinate (bytes) of the packed box of K block kb: 16-byte aligned, as TMA requires.
template <int OPA>
__device__ __forceinline__ int dec_box_x(int kb) {
  return OPA == OPA_U8 ? kb * 32 : (kb >> 1) * 16;
}

// Raster: tiles go down group_m m-tiles (markers) first, then across the n-tiles (phenotypes),
// so the tiles in flight at once share a few A stripes and a band of B stripes in L2.
__device__ __forceinline__ void tile_coord(int tile, int n_mt, int n_nt, int group_m, int& mt,
                                           int& nt) {
  const int group = group_m * n_nt;
  const int g = tile / group;
  const int first = g * group_m;
  const int gm = min(group_m, n_mt - first);
  const int idx = tile - g * group;
  mt = first + idx % gm;
  nt = idx / gm;
}

// Statistics of the 128 totals one thread holds: its marker row against 128 consecutive
// phenotype columns starting at col0, in groups of 16 columns.
// D of a column is tot + shift * col_cs[col] (the marker row was shifted by `shift`).
// Per column: r, the hit test, optionally every statistic's r, and the column's best marker
// over the warp's 32 rows: one warp max (redux.sync) of the ordered key bits(|r|) + 1 (0 for
// NaN; non-negative floats order like their bits), the lowest lane holding it (the smallest
// marker) offering it to the global per-phenotype best.
// The 128 columns go in 8 rolled groups of 16, the totals shifted down by 16 registers after
// each group: fully unrolled, this runs once per tile through tens of KB of straight-line code
// and stalls on instruction fetch long enough to hold up the products.
__device__ __forceinline__ void epilogue_tile(const EpiParams& ep, float (&tot)[128],
                                              long long row, long long row_base, bool row_ok,
                                              float rinv, float shift, int col0, int lane) {
#pragma unroll 1
  for (int g = 0; g < 8; ++g) {
    // keys of the group's 16 columns, then 16 independent warp maxima, then the ballots: the
    // collective operations of different columns overlap instead of forming one chain
    uint32_t u[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int col = col0 + 16 * g + k;
      float r = __int_as_float(0x7fc00000);
      if (row_ok && col < ep.P) {
        const float D = fmaf(shift, ep.col_cs[col], tot[k]);
        r = corr_nan(D, rinv, ep.col_rmul[col]);
        if (ep.do_hits && r * r >= ep.r2_thr) emit_hit_raw(ep, D, row, col);
        if (ep.do_full) ep.rstore[row * ep.ldo + col] = r;
      }
      u[k] = (r == r) ? __float_as_uint(fabsf(r)) + 1u : 0u;
    }
    if (ep.do_best) {
      uint32_t cmax[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) cmax[k] = __reduce_max_sync(0xffffffffu, u[k]);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (!cmax[k]) continue;  // warp-uniform
        const uint32_t owners = __ballot_sync(0xffffffffu, u[k] == cmax[k]);
        if (lane == __ffs(owners) - 1) {
          const long long marker = ep.marker_offset + row_base + lane;
          best_offer(ep.best + col0 + 16 * g + k,
                     ((unsigned long long)(u[k] - 1u) << 32) |
                         (unsigned long long)(0xFFFFFFFFu - (uint32_t)marker));
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 112; ++i) tot[i] = tot[i + 16];
  }
}

}  // namespace tcx
}  // namespace tg
