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
//                  of 64 bytes per row with the 64-byte swizzle for dosages, 16 bytes for 2-bit
//                  calls; 256 or 128 rows) into a ring of its own, kept PS - 1 stages ahead of
//                  the decoders, and the joint B operand's hi and lo halves for each stage into
//                  the B ring
//   warp 1 lane 0  MMA issuer: per stage 2 K blocks x 2 k-steps x MS sub-tiles x 2 products
//                  (hi, lo) of tcgen05.mma 128 x bn x 16 with A read from tensor memory,
//                  accumulation chunked as in k_tc_scan (a fresh accumulator per 1024 samples,
//                  two accumulators alternating)
//   warps 4..11    decoders, then epilogue: thread = one tile row = one TMEM lane (MS = 2: 256
//                  rows, both K blocks of a stage; MS = 1: 128 rows, the two column halves of
//                  warps taking one K block each). Each stage they expand their row from the
//                  packed slot (genotype.cuh: code - c exactly, bf16(mean - c) for a missing call,
//                  0 past N) and write it straight into the stage's A columns of tensor memory
//                  with tcgen05.st (32 or 16 columns of their lane), so A never passes through
//                  shared memory and needs no proxy fence: tcgen05.wait::st and the tcgen05
//                  thread-sync fence order it before the stage's full barrier. After the last
//                  stage of each chunk they drain the chunk before it (tcgen05.ld) into FP32
//                  totals in registers; at the end of a tile they drain its last chunk and write
//                  their row's raw products D + c * sum_i B (as k_tc_scan's raw mode).
// The projection of a larger panel (P + q - 1 > 128) runs as the same pass with the 64
// projection columns alone; there the decoders also write the block's bf16 operand for the
// panel's contraction as they expand each stage (staged per warp in shared memory so that each
// store instruction writes whole 128-byte row segments). The operand is then written once and
// read once, by the contraction, and the projection reads the packed rows instead of it.
// TMEM: the two chunk accumulators (MS x bn columns each) from column 0, four A stages of
// MS x 32 columns (two 16-bit values per column) from column 256. The 128-column pass on
// 256-marker tiles cannot fit its A stages there and keeps A in shared memory
// (k_joint_fused_sm below).
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

// Register split of the joint passes: warpgroup 0 holds only the producer and the MMA issuer
// (warps 2-3 idle; the epilogue warps decode), so it gives back down to 56 registers and the two
// epilogue warpgroups take 224: 128 x 56 + 256 x 224 = 64,512, the launch total (384 x 168).
constexpr int kJointLow = 56, kJointHigh = 224;
static_assert(128 * kJointLow + 256 * kJointHigh <= kThreads * 168, "register split exceeds launch");

template <int OPA, int BR, int MS>
struct FCfg {
  static constexpr int kRows = MS * TBM;                          // tile rows
  static constexpr int kBoxP = OPA == OPA_U8 ? 64 : 16;            // packed bytes per row per stage
  static constexpr int kPackBytes = kRows * kBoxP;                 // one packed slot
  static constexpr int kBk = BR * TBK * 2;                         // one K block of B rows
  static constexpr int kStageBytes = 4 * kBk;                      // Bhi, Blo of 2 K blocks
  static constexpr int kPS = 8;                                    // packed ring slots
  static constexpr int kStages = 4;                                // B ring slots = A stages in TMEM
  // TMEM: two chunk accumulators of MS x BR columns at 0 and MS x BR, then the A stages from
  // column 256, MS x 32 columns each (a row's 64 samples, two 16-bit values per column)
  static constexpr int kAccCols = MS * BR;
  static constexpr int kACol = 256;
  static constexpr int kAStageCols = MS * 32;
  static_assert(2 * kAccCols <= kACol && kACol + kStages * kAStageCols <= kTmemCols, "TMEM");
  static constexpr int kBarBytes = 256;
  // the operand write (64-column pass): each decoder warp stages its 32 rows of a stage (MS x 64
  // bytes each) so that its global stores cover whole rows' segments
  static constexpr int kStgRow = MS * 64;
  static constexpr int kStgBytes = BR == 64 ? kEpiWarps * 32 * kStgRow : 0;
  static constexpr int kSmem =
      kStages * kStageBytes + kPS * kPackBytes + kBarBytes + kStgBytes + 1024;
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

// 16 dosage bytes v minus the row's shift c as f16 pairs, exactly: byte b placed under the f16
// exponent of 1024 is the f16 value 1024 + b (bits 0x6400 | b, one byte permute per pair), and
// one f16x2 subtraction of 1024 + c (c an integer in [0, 255]) leaves b - c, exact in f16.
__device__ __forceinline__ void split16_u8_f16(uint4 v, uint32_t c2, uint32_t* o) {
  const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint32_t h = __byte_perm(w4[p >> 1], 0x64646464u, (p & 1) ? 0x4342u : 0x4140u);
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(o[p]) : "r"(h), "r"(c2));
  }
}

// Zero the 16-bit values of samples >= N among the 16 starting at i0 (8 words).
__device__ __forceinline__ void zero_tail16p(uint32_t* o, int i0, int N) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int i = i0 + 2 * p;
    if (i >= N) o[p] = 0u;
    else if (i + 1 >= N) o[p] &= 0xFFFFu;
  }
}

// Store 32 consecutive TMEM columns of this thread's lane (the warp's 32 lanes at once).
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
      "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]),
      "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]),
      "r"(v[30]), "r"(v[31])
      : "memory");
}
__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// A from tensor memory: D (+)= A[a_tmem] B[b_desc]^T.
__device__ __forceinline__ void tc_mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Sum and sum of squares of 16 dosage bytes whose first sample is i0, the samples >= N left out
// (past N the packed row holds the caller's padding).
__device__ __forceinline__ void sums16_u8(uint4 v, int i0, int N, uint32_t& s, uint32_t& s2) {
  const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
  if (i0 + 16 <= N) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s = __dp4a(w4[q], 0x01010101u, s);
      s2 = __dp4a(w4[q], w4[q], s2);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t u = (w4[q] >> (8 * b)) & 0xFFu;
        if (i0 + 4 * q + b < N) {
          s += u;
          s2 += u * u;
        }
      }
  }
}

// A dosage row's shift taken from its first packed slot (samples 0..63, 64-byte swizzle): the
// rounded mean of its first min(N, 64) bytes. Any integer shift leaves b - c exact in f16; one
// near the row's mean keeps the partial sums of the products small, as the full mean does.
__device__ __forceinline__ uint32_t first_slot_shift_u8(uint32_t src, int r, int N) {
  const uint32_t sw = (uint32_t)((r >> 1) & 3);
  uint32_t s = 0, s2 = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if (16 * g >= N) break;
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(src + ((((uint32_t)g) ^ sw) << 4)));
    sums16_u8(v, 16 * g, N, s, s2);
  }
  const int n = N < 64 ? N : 64;
  const int c = (int)rintf((float)s / (float)n);
  return (uint32_t)(c < 0 ? 0 : c > 255 ? 255 : c);
}

// A dosage row's statistics from its exact byte sums, as the counting pass writes them: n_obs =
// N (no mask), mean = S / N, |g_c|^2 = (N S2 - S^2) / N (the numerator exact in 64-bit
// integers), and the shift the row was expanded with. S2 <= 255^2 N fits 32 bits for
// N <= 66,051, the limit of this form.
__device__ __forceinline__ void write_row_stats(const DecodeArgs& da, long long row, uint32_t c,
                                                uint32_t S, uint32_t S2) {
  const double dn = (double)da.N;
  da.nobs_out[row] = da.N;
  da.mean_out[row] = (double)S / dn;
  const long long num = (long long)S2 * (long long)da.N - (long long)S * (long long)S;
  da.gc2_out[row] = (double)num / dn;
  da.shift_out[row] = (float)c;
}

// Expand `n16` groups of 16 samples of one row, starting at sample i0, from the packed slot
// (row base `src`, shared) into o (8 words per group): 2-bit calls as bf16 (k = the row's lookup
// pair), dosage bytes as f16 (k.x = the f16 pair of 1024 + c). Dosage slots carry the TMA's
// 64-byte swizzle (16-byte chunk j of row r at r * 64 + 16 * (j ^ ((r >> 1) & 3))), so the 8
// threads of a quarter warp, 8 consecutive rows, read 8 distinct bank groups. Dosage bytes are
// also added into s and s2 (their sum and sum of squares, samples < N only).
template <int OPA>
__device__ __forceinline__ void expand_groups(uint32_t src, int r, int g0, int n16, uint2 k,
                                              bool row_ok, int i0, int N, uint32_t* o,
                                              uint32_t& s, uint32_t& s2) {
  if (OPA == OPA_2BIT) {
    uint32_t w[4];
    if (n16 == 4) {
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                   : "r"(src));
    } else {
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(src + 4 * g0));
    }
#pragma unroll
    for (int g = 0; g < 4; ++g)
      if (g < n16) split16_2bit(w[g], k.x, k.y, *reinterpret_cast<uint32_t(*)[8]>(o + 8 * g));
  } else {
    const uint32_t sw = (uint32_t)((r >> 1) & 3);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g >= n16) break;
      uint4 v;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                   : "r"(src + ((((uint32_t)(g0 + g)) ^ sw) << 4)));
      split16_u8_f16(v, k.x, o + 8 * g);
      sums16_u8(v, i0 + 16 * g, N, s, s2);
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if (g >= n16) break;
    if (!row_ok) {
#pragma unroll
      for (int p = 0; p < 8; ++p) o[8 * g + p] = 0u;
    } else if (i0 + 16 * g + 16 > N) {
      zero_tail16p(o + 8 * g, i0 + 16 * g, N);
    }
  }
}

// Write a stage of the block's bf16 operand from the expanded rows of one decoder warp: lane l
// holds row l of the warp's 32 (NW words, two 16-bit values each, NW = 32: 64 samples, or 16:
// 32 samples). The rows go through the warp's staging area in shared memory (`stg`, 32 rows of
// 4 NW bytes; 16-byte chunk c of row l at chunk c ^ swz(l), which keeps each quarter warp on
// distinct banks both ways), then each store instruction writes 4 rows of 128 bytes (NW = 32) or
// 8 rows of 64 bytes (NW = 16), whole segments, instead of 32 scattered 16-byte pieces. Row l
// goes to dst0 + l * ld (16-byte aligned); rows at or past `rows` are skipped.
// 2-bit values are bf16 already. Dosage values are f16 of b - c, integers of magnitude at most
// 255 (or 0 past N), which bf16 holds exactly, so the conversion through f32 is exact and gives
// the decoded operand's bits.
template <int OPA, int NW>
__device__ __forceinline__ void store_operand_warp(uint32_t stg, const uint32_t* o, int lane,
                                                   __nv_bfloat16* dst0, long long ld, int rows) {
  constexpr int kChunks = NW / 4;          // 16-byte chunks per row
  constexpr int kRowB = NW * 4;            // bytes per row
  constexpr int kRowsPer = 32 / kChunks;   // rows per store instruction
  auto swz = [](int r) { return kChunks == 8 ? (r & 7) : ((r >> 1) & 3); };
  __syncwarp();  // the previous stage's staged rows have been read
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t x = o[4 * c + i];
      if (OPA == OPA_U8) {
        __half2 h;
        memcpy(&h, &x, 4);
        const __nv_bfloat162 b = __float22bfloat162_rn(__half22float2(h));
        memcpy(&x, &b, 4);
      }
      w[i] = x;
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                     stg + (uint32_t)(lane * kRowB + ((c ^ swz(lane)) << 4))),
                 "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
  }
  __syncwarp();
  const int cc = lane % kChunks;
#pragma unroll
  for (int i = 0; i < 32 / kRowsPer; ++i) {
    const int r = i * kRowsPer + lane / kChunks;
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(stg + (uint32_t)(r * kRowB + ((cc ^ swz(r)) << 4))));
    if (r < rows) *reinterpret_cast<uint4*>(dst0 + r * ld + cc * 8) = v;
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
  const uint32_t stg_base = bars + C::kBarBytes;  // the operand write's staging rows

  auto sBhi = [&](int s, int h) { return base + (uint32_t)(s * C::kStageBytes + h * C::kBk); };
  auto sBlo = [&](int s, int h) {
    return base + (uint32_t)(s * C::kStageBytes + 2 * C::kBk + h * C::kBk);
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

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kJointLow));
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
      // ---------------------------------------------------------- MMA issuer (A from TMEM)
      // A and B both bf16 (2-bit calls) or both f16 (dosage bytes, scaled f16 joint operand)
      const uint32_t idesc = OPA == OPA_U8 ? idesc_f16(BR) : idesc_bf16(BR);
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
          const uint32_t d = tmem_base + (uint32_t)(acc * C::kAccCols);
          const int kb1 = chunk_end(kb0, num_kb);
          for (int kb = kb0; kb < kb1; kb += 2, ++j) {
            const int s = j % S;
            if (!mbar_wait(full_bar(s), (uint32_t)((j / S) & 1), abort_flag, spin_ns, ep.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_stage = tmem_base + (uint32_t)(C::kACol + s * C::kAStageCols);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int k = 0; k < TBK / 16; ++k) {
                const uint64_t bh = sdesc_sw64(sBhi(s, h) + 32u * k);
                const uint64_t bl = sdesc_sw64(sBlo(s, h) + 32u * k);
#pragma unroll
                for (int sub = 0; sub < MS; ++sub) {
                  // 16 samples = 8 columns of the sub-tile's 32 (K block h, k-step k)
                  const uint32_t a = a_stage + (uint32_t)(sub * 32 + h * 16 + k * 8);
                  const uint32_t ds = d + (uint32_t)(sub * BR);
                  tc_mma_ta(ds, a, bh, idesc, (kb > kb0 || h > 0 || k > 0) ? 1u : 0u);
                  tc_mma_ta(ds, a, bl, idesc, 1u);
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
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kJointHigh));
    // ------------------------------------------------------------ decoders, then epilogue
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;
    // MS = 2: tile row half * 128 + quarter * 32 + lane (TMEM lane quarter * 32 + lane of
    // sub-tile `half`), both K blocks of a stage; MS = 1: tile row quarter * 32 + lane, K block
    // `half` of each stage
    const int rr = quarter * 32 + lane;
    const int trow = (MS == 2 ? half * 128 : 0) + rr;
    const int sub = MS == 2 ? half : 0;
    const bool drains = MS == 2 || half == 0;     // MS = 1: columns [0, BR) sit in half 0's warps
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    int j = 0;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
      const int mt = (int)blockIdx.x + t * (int)gridDim.x;
      const long long row = (long long)mt * C::kRows + trow;
      const bool row_ok = row < ep.M;
      // one pass (dosage rows on 256-row tiles, statistics written here): the row's shift comes
      // from the tile's first packed slot, in the first stage
      const bool one_pass = OPA == OPA_U8 && MS == 2 && da.shift_out != nullptr;
      uint32_t c_row = 0;
      uint2 kc = make_uint2(0u, 0u);
      if (OPA == OPA_2BIT) {
        kc = dec_row_consts<OPA>(da, row);
      } else if (!one_pass) {  // the f16 pair of 1024 + c (c = the row's integer shift)
        c_row = row_ok ? (uint32_t)da.shift[row] : 0u;
        const uint32_t c16 = 0x6400u + c_row;
        kc = make_uint2(c16 | (c16 << 16), 0u);
      }
      uint32_t sum1 = 0, sum2 = 0;  // the row's bytes and their squares (dosage; N <= 66,051)
      float tot[BR];
#pragma unroll
      for (int e = 0; e < BR; ++e) tot[e] = 0.0f;
      auto drain = [&](uint32_t c) -> bool {
        const int acc = (int)(c & 1u);
        if (!mbar_wait(cfull_bar(acc), (c >> 1) & 1u, abort_flag, spin_ns, ep.status)) return false;
        tc_fence_after();
        if (drains) {
          const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * C::kAccCols + sub * BR);
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
          tc_fence_after();  // the products that read this A stage have completed
          const uint32_t src = sPk(p) + (uint32_t)(trow * C::kBoxP);
          if (one_pass && kb == 0) {
            c_row = row_ok ? first_slot_shift_u8(src, trow, da.N) : 0u;
            const uint32_t c16 = 0x6400u + c_row;
            kc = make_uint2(c16 | (c16 << 16), 0u);
          }
          uint32_t o[32];
          uint32_t s1 = 0, s2 = 0;
          const uint32_t a_row = tmem_base + lane_addr + (uint32_t)(C::kACol + s * C::kAStageCols);
          if (MS == 2) {  // the row's 64 samples: 32 columns of sub-tile `half`
            expand_groups<OPA>(src, trow, 0, 4, kc, row_ok, kb * TBK, da.N, o, s1, s2);
            sum1 += s1;
            sum2 += s2;
            __syncwarp();
            if (lane == 0) mbar_arrive(pempty_bar(p));  // the packed slot is read
            tc_st32(a_row + (uint32_t)(sub * 32), o);
          } else {  // K block `half`: 32 samples, 16 columns
            expand_groups<OPA>(src, trow, 2 * half, 2, kc, row_ok, (kb + half) * TBK, da.N, o, s1,
                               s2);
            __syncwarp();
            if (lane == 0) mbar_arrive(pempty_bar(p));
            tc_st16(a_row + (uint32_t)(half * 16), o);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(full_bar(s));
          // the projection pass of a larger panel: the expanded rows are also the block's operand
          if (da.a_out != nullptr) {
            const long long row0 = row - lane;  // the warp's first row
            const int rows = ep.M - row0 < 32 ? (int)(ep.M - row0) : 32;
            __nv_bfloat16* dst0 =
                da.a_out + row0 * da.lda_out + (long long)(MS == 2 ? kb : kb + half) * TBK;
            const uint32_t stg = stg_base + (uint32_t)((warp - 4) * 32 * C::kStgRow);
            if (MS == 2) store_operand_warp<OPA, 32>(stg, o, lane, dst0, da.lda_out, rows);
            else store_operand_warp<OPA, 16>(stg, o, lane, dst0, da.lda_out, rows);
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
      if (one_pass && row_ok) write_row_stats(da, row, c_row, sum1, sum2);
      // the tile's raw products: the first raw_cols columns, unnormalised, with the shift's
      // add-back
      if (drains && row_ok) {
        const float shift = one_pass ? (float)c_row : ep.row_shift ? ep.row_shift[row] : 0.0f;
        // the f16 joint operand holds 2^14 v (an exact power of two to take back)
        constexpr float kUnscale = OPA == OPA_U8 ? (float)(1.0 / kJointF16Scale) : 1.0f;
#pragma unroll
        for (int e = 0; e < BR; ++e)
          if (e < ep.raw_cols)
            ep.raw_out[row * ep.raw_ld + e] = fmaf(shift, ep.col_cs[e], tot[e]) * kUnscale;
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

// The 128-column pass on 256-marker tiles keeps A in shared memory: its two accumulators (two
// sub-tiles of 128 columns, double-buffered) fill all 512 TMEM columns. Same roles and barriers
// as k_joint_fused, except that the decoders store their expanded row into the stage's two
// 64-byte-swizzled A tiles (one per K block; 16-byte chunk j of row rr at
// rr * 64 + 16 * (j ^ ((rr >> 1) & 3)), where the operand's TMA would put it), fence them for the
// async proxy once per stage, and the products read A through shared-memory descriptors.
template <int OPA>
struct SCfg {
  static constexpr int kRows = 2 * TBM;
  static constexpr int kBoxP = OPA == OPA_U8 ? 64 : 16;
  static constexpr int kPackBytes = kRows * kBoxP;
  static constexpr int kAk = 2 * A_BYTES;                          // one K block of both sub-tiles
  static constexpr int kBk = 128 * TBK * 2;
  static constexpr int kStageBytes = 2 * kAk + 4 * kBk;            // A (2 K blocks), Bhi, Blo
  static constexpr int kStages = 2;
  static constexpr int kPS0 = (210 * 1024 - kStages * kStageBytes) / kPackBytes;
  static constexpr int kPS = kPS0 > 8 ? 8 : kPS0;
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStageBytes + kPS * kPackBytes + kBarBytes + 1024;
  static_assert(kPS >= 2 && kSmem <= 227 * 1024, "shared memory");
};

template <int OPA>
__global__ void __launch_bounds__(kThreads, 1)
    k_joint_fused_sm(const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                     int num_kb, int n_mt, long long spin_ns, EpiParams ep,
                     const __grid_constant__ DecodeArgs da) {
  using C = SCfg<OPA>;
  constexpr int S = C::kStages, PS = C::kPS, BR = 128;
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
      mbar_init(full_bar(s), 1 + kEpiWarps);
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
  const int total = my_tiles * stages_per_tile;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kJointLow));
    if (warp == 0 && lane == 0) {
      // ---------------------------------------------------------- TMA producer
      auto load_packed = [&](int j) -> bool {
        const int p = j % PS;
        if (!mbar_wait(pempty_bar(p), (uint32_t)((j / PS) & 1) ^ 1u, abort_flag, spin_ns, ep.status))
          return false;
        const int mt = (int)blockIdx.x + (j / stages_per_tile) * (int)gridDim.x;
        mbar_expect_tx(pfull_bar(p), (uint32_t)C::kPackBytes);
        tma_load_2d(&da.tmG, sPk(p), pfull_bar(p), (j % stages_per_tile) * C::kBoxP, mt * C::kRows);
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
        if (!mbar_wait(empty_bar(s), (uint32_t)((j / S) & 1) ^ 1u, abort_flag, spin_ns, ep.status)) {
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
      for (int j = total - S > 0 ? total - S : 0; j < total; ++j)
        mbar_wait(full_bar(j % S), (uint32_t)((j / S) & 1), abort_flag, spin_ns, ep.status);
      for (int j = total - PS > 0 ? total - PS : 0; j < total; ++j)
        mbar_wait(pfull_bar(j % PS), (uint32_t)((j / PS) & 1), abort_flag, spin_ns, ep.status);
    } else if (warp == 1 && lane == 0) {
      // ---------------------------------------------------------- MMA issuer (A in shared memory)
      const uint32_t idesc = OPA == OPA_U8 ? idesc_f16(BR) : idesc_bf16(BR);
      uint32_t g = 0;
      int j = 0;
      bool ok = true;
      for (int t = 0; t < my_tiles && ok; ++t) {
        for (int kb0 = 0; kb0 < num_kb && ok; kb0 = chunk_end(kb0, num_kb), ++g) {
          const int acc = (int)(g & 1u);
          if (!mbar_wait(cempty_bar(acc), ((g >> 1) & 1u) ^ 1u, abort_flag, spin_ns, ep.status)) {
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
                for (int sub = 0; sub < 2; ++sub) {
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
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kJointHigh));
    // ------------------------------------------------------------ decoders, then epilogue
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;  // sub-tile
    const int rr = quarter * 32 + lane;
    const int trow = half * 128 + rr;
    const uint32_t sw = (uint32_t)((rr >> 1) & 3);
    uint32_t g = 0;
    int j = 0;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
      const int mt = (int)blockIdx.x + t * (int)gridDim.x;
      const long long row = (long long)mt * C::kRows + trow;
      const bool row_ok = row < ep.M;
      // one pass (dosage rows, statistics written here): the shift from the first packed slot
      const bool one_pass = OPA == OPA_U8 && da.shift_out != nullptr;
      uint32_t c_row = 0;
      uint2 kc = make_uint2(0u, 0u);
      if (OPA == OPA_2BIT) {
        kc = dec_row_consts<OPA>(da, row);
      } else if (!one_pass) {
        c_row = row_ok ? (uint32_t)da.shift[row] : 0u;
        const uint32_t c16 = 0x6400u + c_row;
        kc = make_uint2(c16 | (c16 << 16), 0u);
      }
      uint32_t sum1 = 0, sum2 = 0;  // the row's bytes and their squares (dosage; N <= 66,051)
      float tot[BR];
#pragma unroll
      for (int e = 0; e < BR; ++e) tot[e] = 0.0f;
      auto drain = [&](uint32_t c) -> bool {
        const int acc = (int)(c & 1u);
        if (!mbar_wait(cfull_bar(acc), (c >> 1) & 1u, abort_flag, spin_ns, ep.status)) return false;
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(acc * TBN + half * 128);
#pragma unroll
        for (int i = 0; i < BR / 32; ++i) {
          float v[32];
          __syncwarp();
          tc_ld32(taddr + (uint32_t)(i * 32), v);
#pragma unroll
          for (int e = 0; e < 32; ++e) tot[i * 32 + e] += v[e];
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
          if (one_pass && kb == 0) {
            c_row = row_ok ? first_slot_shift_u8(src, trow, da.N) : 0u;
            const uint32_t c16 = 0x6400u + c_row;
            kc = make_uint2(c16 | (c16 << 16), 0u);
          }
          uint32_t s1 = 0, s2 = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // one K block (32 samples, 64 bytes of the row) at a time
            uint32_t o[16];
            expand_groups<OPA>(src, trow, 2 * h, 2, kc, row_ok, (kb + h) * TBK, da.N, o, s1, s2);
            const uint32_t row_base = sA(s, h, half) + (uint32_t)rr * 64u;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                               row_base + ((((uint32_t)c) ^ sw) << 4)),
                           "r"(o[4 * c]), "r"(o[4 * c + 1]), "r"(o[4 * c + 2]), "r"(o[4 * c + 3])
                           : "memory");
          }
          sum1 += s1;
          sum2 += s2;
          __syncwarp();
          if (lane == 0) mbar_arrive(pempty_bar(p));  // the packed slot is read
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
          __syncwarp();
          if (lane == 0) mbar_arrive(full_bar(s));
        }
        if (!ok) break;
        if (g > g_first && !drain(g - 1)) {
          ok = false;
          break;
        }
      }
      if (!ok || !drain(g - 1)) {
        ok = false;
        break;
      }
      if (one_pass && row_ok) write_row_stats(da, row, c_row, sum1, sum2);
      if (row_ok) {
        const float shift = one_pass ? (float)c_row : ep.row_shift ? ep.row_shift[row] : 0.0f;
        constexpr float kUnscale = OPA == OPA_U8 ? (float)(1.0 / kJointF16Scale) : 1.0f;
#pragma unroll
        for (int e = 0; e < BR; ++e)
          if (e < ep.raw_cols)
            ep.raw_out[row * ep.raw_ld + e] = fmaf(shift, ep.col_cs[e], tot[e]) * kUnscale;
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

template <int OPA>
cudaError_t go_fused_sm(const CUtensorMap* bh, const CUtensorMap* bl, int64_t K, const EpiParams& ep,
                        int sm_count, long long spin_ns, cudaStream_t st, const DecodeArgs& da) {
  using C = SCfg<OPA>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_joint_fused_sm<OPA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + C::kRows - 1) / C::kRows;
  const int grid = n_mt < sm_count ? n_mt : sm_count;
  k_joint_fused_sm<OPA><<<grid, kThreads, C::kSmem, st>>>(*bh, *bl, (int)(K / TBK), n_mt, spin_ns,
                                                           ep, da);
  return cudaGetLastError();
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

int joint_fused_rows(int64_t M, int sm_count, int joint_cols) {
  (void)joint_cols;  // both widths take 256-marker tiles once those fill every SM at least once
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
  const int jc = ep.raw_cols <= 64 ? 64 : 128;
  const bool two = joint_fused_rows(ep.M, sm_count, jc) == 2 * TBM;
  const bool u8 = encoding == TG_ENC_U8_DOSAGE;
  // the one-pass statistics need a thread per row: dosage rows on 256-row tiles
  if (da.shift_out && (!u8 || !two || da.N > kOnePassMaxN || !da.nobs_out || !da.mean_out ||
                       !da.gc2_out))
    return cudaErrorInvalidValue;
  // the operand write: the 64-column pass (A in tensor memory), every column of a row in
  // 16-byte stores
  if (da.a_out && (jc != 64 || da.lda_out < K || da.lda_out % 8 ||
                   reinterpret_cast<uintptr_t>(da.a_out) % 16))
    return cudaErrorInvalidValue;
  if (jc == 64) {  // A in tensor memory
    if (u8) return two ? go_fused<OPA_U8, 64, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
                       : go_fused<OPA_U8, 64, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
    return two ? go_fused<OPA_2BIT, 64, 2>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
               : go_fused<OPA_2BIT, 64, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
  }
  if (two)  // 128 columns on 256-marker tiles: A in shared memory
    return u8 ? go_fused_sm<OPA_U8>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
              : go_fused_sm<OPA_2BIT>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
  return u8 ? go_fused<OPA_U8, 128, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da)
            : go_fused<OPA_2BIT, 128, 1>(tmBhi, tmBlo, K, ep, sm_count, spin_ns, st, da);
}

}  // namespace tg
