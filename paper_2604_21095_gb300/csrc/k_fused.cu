// The projection pass of a small panel with the genotype decode fused into it (Section 2.2: the
// covariate projection of each marker and Eq. 2 for a panel of P <= 128 - (q - 1) phenotypes,
// read from the packed genotype block in one pass; Section 2.4: the scan is bound by the bytes it
// reads).
//
// For a small panel the whole scan is one pass over the block: the joint B operand holds the
// q - 1 covariate projection columns and the P phenotype columns (64 or 128 rows), so a single
// contraction gives both Q^T a and the panel's products. With the decoded operand in HBM that
// pass reads 2 bytes per sample and marker after the decode wrote them; here it reads the packed
// rows instead (1 byte per sample for dosages, 1/4 for 2-bit calls) and expands them in shared
// memory, which removes the operand's round trip through HBM.
//
// Persistent kernel, one CTA per SM, 384 threads:
//   warp 0 lane 0  TMA producer: the packed rows of each stage (two K blocks, 64 samples: a box
//                  of 64 bytes per row for dosages, 16 for 2-bit calls, 256 or 128 rows) into a
//                  ring of its own, kept PS - 1 stages ahead of the decoders, and the joint B
//                  operand's hi and lo halves for each stage into the A/B stage ring
//   warp 1 lane 0  MMA issuer: per stage 2 K blocks x 2 k-steps x MS sub-tiles x 2 products
//                  (hi, lo) of tcgen05.mma 128 x bn x 16, accumulation chunked as in k_tc_scan
//                  (a fresh accumulator per 1024 samples, two accumulators alternating)
//   warps 4..11    decoders, then epilogue: thread = one tile row (MS = 2: 256 rows, one per
//                  thread, both K blocks of a stage; MS = 1: 128 rows, the two column halves of
//                  warps taking one K block each). Each stage they expand their row from the
//                  packed slot into the 64-byte-swizzled A tile (genotype.cuh: code - c exactly,
//                  bf16(mean - c) for a missing call, 0 past N), fence the stores for the async
//                  proxy once, and join the stage's full barrier; after the last stage of each
//                  chunk they drain the chunk before it (tcgen05.ld of their TMEM lane) into
//                  FP32 totals in registers, and at the end of a tile they drain its last chunk
//                  and write their row's raw products D + c * sum_i B (as k_tc_scan's raw mode).
// The A values, the products and their order are those of k_tc_scan on the decoded operand, so
// the results are bit-identical to it. The per-marker shift c and missing value come from the
// counting pass of the decode (launch_decode without an operand).
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

template <int OPA, int BR, int MS>
struct FCfg {
  static constexpr int kRows = MS * TBM;                          // tile rows
  static constexpr int kBoxP = OPA == OPA_U8 ? 64 : 16;            // packed bytes per row per stage
  static constexpr int kPackBytes = kRows * kBoxP;                 // one packed slot
  static constexpr int kAk = MS * A_BYTES;                         // one K block of A
  static constexpr int kBk = BR * TBK * 2;                         // one K block of B rows
  static constexpr int kStageBytes = 2 * kAk + 4 * kBk;            // A (2 K blocks), Bhi, Blo
  static constexpr int kBudget = 210 * 1024;
  static constexpr int kPS = OPA == OPA_U8 ? 4 : 8;                // packed ring slots
  static constexpr int kS0 = (kBudget - kPS * kPackBytes) / kStageBytes;
  static constexpr int kStages = kS0 > 4 ? 4 : kS0;                // A/B ring slots
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStageBytes + kPS * kPackBytes + kBarBytes + 1024;
  static_assert(kStages >= 2, "at least two A/B stages");
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

// Expand K block kb (32 samples) of one row from its packed bytes `src` (shared) into the row's
// 64 bytes of an A tile (shared, 64-byte swizzle: 16-byte chunk j of row rr at
// rr * 64 + 16 * (j ^ ((rr >> 1) & 3))).
template <int OPA>
__device__ __forceinline__ void expand_kblock(uint32_t src, uint2 k, bool row_ok, int rr, int kb,
                                              int N, uint32_t a_tile) {
  const uint32_t row_base = a_tile + (uint32_t)rr * 64u;
  const uint32_t sw = (uint32_t)((rr >> 1) & 3);
#pragma unroll
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

template <int OPA, int BR, int MS>
__global__ void __launch_bounds__(kThreads, 1)
    k_joint_fused(const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                  int num_kb, int n_mt, long long spin_ns, EpiParams ep,
                  const __grid_constant__ DecodeArgs da) {
  using C = FCfg<OPA, BR, MS>;
  constexpr int S = C::kStages, PS = C::kPS;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t pk_base = base + S * C::kStageBytes;
  const uint32_t bars = pk_base + PS * C::kPackBytes;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (S + s); };
  auto pfull_bar = [&](int p) { return bars + 8u * (2 * S + p); };
  auto pempty_bar = [&](int p) { return bars + 8u * (2 * S + PS + p); };
  auto cfull_bar = [&](int a) { return bars + 8u * (2 * S + 2 * PS + a); };
  auto cempty_bar = [&](int a) { return bars + 8u * (2 * S + 2 * PS + 2 + a); };
  const uint32_t drain_bar = bars + 8u * (2 * S + 2 * PS + 4);
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(gbase + (bars - base) + 8 * (2 * S + 2 * PS + 5));
  static_assert(8 * (2 * S + 2 * PS + 5) + 8 <= C::kBarBytes, "barrier area");
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  auto sA = [&](int s, int h, int sub) {
    return base + (uint32_t)(s * C::kStageBytes + h * C::kAk + sub * A_BYTES);
  };
  auto sBhi = [&](int s, int h) {
    return base + (uint32_t)(s * C::kStageBytes + 2 * C::kAk + h * C::kBk);
  };
  auto sBlo = [&](int s, int h) {
    return base + (uint32_t)(s * C::kStageBytes + 2 * C::kAk + 2 * C::kBk + h * C::kBk);
  };
  auto sPk = [&](int p) { return pk_base + (uint32_t)(p * C::kPackBytes); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1 + kEpiWarps);  // the producer's B bytes + one arrival per decoder warp
      mbar_init(empty_bar(s), 1);
    }
    for (int p = 0; p < PS; ++p) {
      mbar_init(pfull_bar(p), 1);
      mbar_init(pempty_bar(p), kEpiWarps);
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
  const int stages_per_tile = num_kb / 2;
  const int my_tiles = blockIdx.x < n_mt ? (n_mt - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * stages_per_tile;  // this CTA's stages, tile after tile
  const int bn = BR;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kLow));
    if (warp == 0 && lane == 0) {
      // ---------------------------------------------------------- TMA producer
      // stage j of this CTA: tile blockIdx.x + (j / stages_per_tile) * gridDim.x, K blocks
      // 2 (j % stages_per_tile) and the next one
      auto load_packed = [&](int j) -> bool {
        const int p = j % PS;
        const uint32_t ph = (uint32_t)((j / PS) & 1);
        if (!mbar_wait(pempty_bar(p), ph ^ 1u, abort_flag, spin_ns, ep.status)) return false;
        const int mt = (int)blockIdx.x + (j / stages_per_tile) * (int)gridDim.x;
        const int st = j % stages_per_tile;
        mbar_expect_tx(pfull_bar(p), (uint32_t)C::kPackBytes);
        tma_load_2d(&da.tmG, sPk(p), pfull_bar(p), st * C::kBoxP, mt * C::kRows);
        return true;
      };
      bool ok = true;
      const int ahead = PS - 1;
      for (int j = 0; j < total && j < ahead && ok; ++j) ok = load_packed(j);
      for (int j = 0; j < total && ok; ++j) {
        if (j + ahead < total && !load_packed(j + ahead)) {
          ok = false;
          break;
        }
        const int s = j % S;
        const uint32_t ph = (uint32_t)((j / S) & 1);
        if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full_bar(s), (uint32_t)(4 * C::kBk));
        const int kb = 2 * (j % stages_per_tile);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tma_load_2d(&tmBhi, sBhi(s, h), full_bar(s), (kb + h) * TBK, 0);
          tma_load_2d(&tmBlo, sBlo(s, h), full_bar(s), (kb + h) * TBK, 0);
        }
      }
      // copies still in flight land before the CTA leaves (bounded)
      for (int j = total - S > 0 ? total - S : 0; j < total; ++j)
        mbar_wait(full_bar(j % S), (uint32_t)((j / S) & 1), abort_flag, spin_ns, ep.status);
      for (int j = total - PS > 0 ? total - PS : 0; j < total; ++j)
        mbar_wait(pfull_bar(j % PS), (uint32_t)((j / PS) & 1), abort_flag, spin_ns, ep.status);
    } else if (warp == 1 && lane == 0) {
      // ---------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16(bn);
      uint32_t g = 0;
      int j = 0;
      bool ok = true;
      for (int t = 0; t < my_tiles && ok; ++t) {
        for (int kb0 = 0; kb0 < num_kb && ok; kb0 = chunk_end(kb0, num_kb), ++g) {
          const int acc = (int)(g & 1u);
          const uint32_t ph = (g >> 1) & 1u;
          if (!mbar_wait(cempty_bar(acc), ph ^ 1u, abort_flag, spin_ns, ep.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(acc * TBN);
          const int kb1 = chunk_end(kb0, num_kb);
          for (int kb = kb0; kb < kb1; kb += 2, ++j) {
            const int s = j % S;
            if (!mbar_wait(full_bar(s), (uint32_t)((j / S) & 1), abort_flag, spin_ns, ep.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int k = 0; k < TBK / 16; ++k) {
                const uint64_t bh = sdesc_sw64(sBhi(s, h) + 32u * k);
                const uint64_t bl = sdesc_sw64(sBlo(s, h) + 32u * k);
#pragma unroll
                for (int sub = 0; sub < MS; ++sub) {
                  const uint64_t a = sdesc_sw64(sA(s, h, sub) + 32u * k);
                  const uint32_t ds = d + (uint32_t)(sub * 128);
                  tc_mma(ds, a, bh, idesc, (kb > kb0 || h > 0 || k > 0) ? 1u : 0u);
                  tc_mma(ds, a, bl, idesc, 1u);
                }
              }
            tc_commit(empty_bar(s));
          }
          if (ok) tc_commit(cfull_bar(acc));
        }
      }
      tc_commit(drain_bar);
      mbar_wait(drain_bar, 0u, abort_flag, spin_ns, ep.status);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RegSplit<OPA>::kHigh));
    // ------------------------------------------------------------ decoders, then epilogue
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;
    // MS = 2: tile row half * 128 + quarter * 32 + lane, sub-tile `half`, both K blocks of a
    // stage; MS = 1: tile row quarter * 32 + lane, K block `half` of each stage
    const int rr = quarter * 32 + lane;           // row within its 128-row sub-tile (TMEM lane)
    const int trow = (MS == 2 ? half * 128 : 0) + rr;
    const int sub = MS == 2 ? half : 0;
    const bool drains = MS == 2 || half == 0;     // MS = 1: columns [0, bn) sit in half 0's warps
    uint32_t g = 0;
    int j = 0;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
      const int mt = (int)blockIdx.x + t * (int)gridDim.x;
      const long long row = (long long)mt * C::kRows + trow;
      const bool row_ok = row < ep.M;
      const uint2 kc = dec_row_consts<OPA>(da, row);
      float tot[BR];
#pragma unroll
      for (int e = 0; e < BR; ++e) tot[e] = 0.0f;
      auto drain = [&](uint32_t c) -> bool {
        const int acc = (int)(c & 1u);
        if (!mbar_wait(cfull_bar(acc), (c >> 1) & 1u, abort_flag, spin_ns, ep.status)) return false;
        tc_fence_after();
        if (drains) {
          const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                 (uint32_t)(acc * TBN + sub * 128);
#pragma unroll
          for (int i = 0; i < BR / 32; ++i) {
            float v[32];
            __syncwarp();
            tc_ld32(taddr + (uint32_t)(i * 32), v);
#pragma unroll
            for (int e = 0; e < 32; ++e) tot[i * 32 + e] += v[e];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(cempty_bar(acc));
        return true;
      };
      const uint32_t g_first = g;
      for (int kb0 = 0; kb0 < num_kb && ok; kb0 = chunk_end(kb0, num_kb), ++g) {
        const int kb1 = chunk_end(kb0, num_kb);
        for (int kb = kb0; kb < kb1; kb += 2, ++j) {
          const int s = j % S, p = j % PS;
          if (!mbar_wait(pfull_bar(p), (uint32_t)((j / PS) & 1), abort_flag, spin_ns, ep.status) ||
              !mbar_wait(empty_bar(s), (uint32_t)((j / S) & 1) ^ 1u, abort_flag, spin_ns, ep.status)) {
            ok = false;
            break;
          }
          const uint32_t src = sPk(p) + (uint32_t)(trow * C::kBoxP);
          if (MS == 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
              expand_kblock<OPA>(src + (uint32_t)(h * (C::kBoxP / 2)), kc, row_ok, rr, kb + h, da.N,
                                 sA(s, h, sub));
          } else {
            expand_kblock<OPA>(src + (uint32_t)(half * (C::kBoxP / 2)), kc, row_ok, rr, kb + half,
                               da.N, sA(s, half, 0));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(full_bar(s));
            mbar_arrive(pempty_bar(p));
          }
        }
        if (!ok) break;
        // the chunk before this one is complete: drain it while the products of this one run
        if (g > g_first && !drain(g - 1)) {
          ok = false;
          break;
        }
      }
      if (!ok || !drain(g - 1)) {  // the tile's last chunk
        ok = false;
        break;
      }
      // the tile's raw products: the first raw_cols columns, unnormalised, with the shift's
      // add-back
      if (drains && row_ok) {
        const float shift = ep.row_shift ? ep.row_shift[row] : 0.0f;
#pragma unroll
        for (int e = 0; e < BR; ++e)
          if (e < ep.raw_cols) ep.raw_out[row * ep.raw_ld + e] = fmaf(shift, ep.col_cs[e], tot[e]);
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

template <int OPA, int BR, int MS>
cudaError_t go_fused(const CUtensorMap* bh, const CUtensorMap* bl, int64_t K, const EpiParams& ep,
                     int sm_count, long long spin_ns, cudaStream_t st, const DecodeArgs& da) {
  using C = FCfg<OPA, BR, MS>;
  static bool attr_set = false;  // per process and instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_joint_fused<OPA, BR, MS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + C::kRows - 1) / C::kRows;
  const int grid = n_mt < sm_count ? n_mt : sm_count;
  k_joint_fused<OPA, BR, MS><<<grid, kThreads, C::kSmem, st>>>(*bh, *bl, (int)(K / TBK), n_mt,
                                                                spin_ns, ep, da);
  return cudaGetLastError();
}

}  // namespace

int joint_fused_rows(int64_t M, int sm_count) {
  return (M + 2 * TBM - 1) / (2 * TBM) >= sm_count ? 2 * TBM : TBM;
}

cudaError_t launch_joint_fused(const CUtensorMap* tmBhi, const CUtensorMap* tmBlo, int64_t K,
                               const EpiParams& ep, int sm_count, long long spin_ns, cudaStream_t st,
                               const DecodeArgs& da, int encoding) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  // raw mode only (the projection, alone or joint with a small panel), 64 or 128 columns,
  // an even number of K blocks, packed rows of the block's M
  if (!ep.raw_out || ep.raw_cols > 128 || ep.P != ep.raw_cols || K % (2 * TBK) || da.M != ep.M ||
      ep.ksplit > 1)
    return cudaErrorInvalidValue;
  const bool two = joint_fused_rows(ep.M, sm_count) == 2 * TBM;
  const bool u8 = encoding == TG_ENC_U8_DOSAGE;
  if (ep.raw_cols <= 64) {
    if (u8) return two ? go_fused<OPA_U8, 64, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
                       : go_fused<OPA_U8, 64, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
    return two ? go_fused<OPA_2BIT, 64, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
               : go_fused<OPA_2BIT, 64, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
  }
  if (u8) return two ? go_fused<OPA_U8, 128, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
                     : go_fused<OPA_U8, 128, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
  return two ? go_fused<OPA_2BIT, 128, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
             : go_fused<OPA_2BIT, 128, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
}

}  // namespace tg
