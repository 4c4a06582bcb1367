// Tensor-core scan: Eq. 2 of Section 2.2 on tcgen05, fused with Eq. 3 and the p-value.
//
// D = A (B_hi + B_lo)^T [+ A_lo B_hi^T] for a block of markers against the whole panel:
//   A     [M][K] bf16  exact genotype codes (or dosage bytes); a missing call holds bf16(mean)
//   A_lo  [M][K] bf16  mean - bf16(mean) at missing calls, 0 elsewhere (2-bit / masked blocks)
//   B_hi, B_lo [P][K]  bf16 split of the unit-norm residualised panel, y ~= hi + lo
// K = samples (zero padded), FP32 accumulation in tensor memory.
//
// Persistent kernel, one CTA per SM, 384 threads (3 warpgroups), warp-specialised:
//   warp 0 lane 0  TMA producer: 128x32 A tiles and 256x32 B tiles (64-byte swizzle) into a
//                  ring of shared-memory stages, completion tracked by mbarrier transaction bytes
//   warp 1 lane 0  MMA issuer: per 32-wide K step, 2 x (2 or 3) tcgen05.mma 128x256x16 into an
//                  FP32 accumulator in TMEM
//   warps 4..11    epilogue: tcgen05.ld of the accumulator (thread = marker row, each warp one
//                  TMEM lane quarter and one half of the 256 columns), r = D / |g_res|, hits
//                  above the r^2 threshold, per-phenotype best marker, optionally every statistic.
// Accumulation is chunked: the tensor core sums at most 512 samples (16 K blocks) into a
// fresh TMEM accumulator, and the epilogue warps add the chunk results into FP32 totals held
// in registers with round-to-nearest adds. The tensor core's FP32 accumulation drops low bits
// toward zero at each chained addition, which over 23,000 samples biases |r| low by about
// 5e-5 relative; chunks of 512 keep that bias near 1e-6. Two chunk accumulators (512 TMEM
// columns) alternate, so draining one overlaps the products of the next.
// Every mbarrier wait is bounded: past the limit the kernel latches ST_TIMEOUT, raises a
// shared abort flag, lets in-flight copies and products finish (again bounded), frees its
// TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

constexpr int TBM = 128, TBN = 256, TBK = 32;  // TBK bf16 = 64 bytes = one swizzle row
constexpr int A_BYTES = TBM * TBK * 2;         // 8 KB
constexpr int B_BYTES = TBN * TBK * 2;         // 16 KB
constexpr int kEpiWarps = 8;
// Three warpgroups: warpgroup 0 = producer warp, MMA warp and two idle warps; warpgroups 1-2 =
// the 8 epilogue warps. At launch every thread gets 168 registers (384 x 168 = 64,512); then
// warpgroup 0 gives registers back (56 each) and the epilogue warpgroups take them
// (224 each): 128 x 56 + 256 x 224 = 64,512, the launch total, so the increase cannot stall.
constexpr int kThreads = 384;
constexpr int kRegsLow = 56;
constexpr int kRegsHigh = 224;
static_assert(128 * kRegsLow + 256 * kRegsHigh <= kThreads * 168, "register split exceeds launch");
constexpr int kTmemCols = 512;                 // two 128 x 256 FP32 chunk accumulators
constexpr int kChunkKB = 16;                   // K blocks per accumulation chunk (512 samples)
constexpr int kGroupM = 8;                     // raster: 8 m-tiles per group

template <bool HAS_LO>
struct Cfg {
  static constexpr int kStageBytes = A_BYTES * (HAS_LO ? 2 : 1) + 2 * B_BYTES;
  static constexpr int kStages = HAS_LO ? 4 : 5;
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStageBytes + kBarBytes + 1024;  // + alignment slack
};

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
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

__device__ __forceinline__ void tile_coord(int tile, int n_mt, int n_nt, int& mt, int& nt) {
  const int group = kGroupM * n_nt;
  const int g = tile / group;
  const int first = g * kGroupM;
  const int gm = min(kGroupM, n_mt - first);
  const int idx = tile - g * group;
  mt = first + idx % gm;
  nt = idx / gm;
}

// Statistics of the 128 totals one thread holds: its marker row against 128 consecutive
// phenotype columns starting at col0, in groups of 16 columns.
__device__ __forceinline__ void epilogue_tile(const EpiParams& ep, const float (&tot)[128],
                                              long long row, long long row_base, bool row_ok,
                                              float rinv, int col0, int lane) {
#pragma unroll
  for (int grp = 0; grp < 8; ++grp) {
    float m[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int col = col0 + grp * 16 + e;
      const float D = tot[grp * 16 + e];
      float r = __int_as_float(0x7fc00000);
      if (row_ok && col < ep.P) r = corr_nan(D, rinv, ep.col_rmul[col]);
      m[e] = (r == r) ? fabsf(r) : -1.0f;
      if (ep.do_hits && r * r >= ep.r2_thr) emit_hit_raw(ep, D, row, col);
      if (ep.do_full && row_ok && col < ep.P) ep.rstore[row * ep.ldo + col] = r;
    }
    if (!ep.do_best) continue;
    // max over the warp's 32 rows: lanes l and l^16 first, then a reduce-scatter over 16
    // lanes after which lane l holds the column max for column grp*16 + (l & 15)
#pragma unroll
    for (int i = 0; i < 16; ++i) m[i] = fmaxf(m[i], __shfl_xor_sync(0xffffffffu, m[i], 16));
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
      const bool upper = (lane & s) != 0;
#pragma unroll
      for (int i = 0; i < s; ++i) {
        const float send = upper ? m[i] : m[i + s];
        const float keep = upper ? m[i + s] : m[i];
        m[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, send, s));
      }
    }
    const float cmax = m[0];
    // the lowest lane (smallest marker) reaching the column max owns the candidate
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float ce = __shfl_sync(0xffffffffu, cmax, e);
      const int col = col0 + grp * 16 + e;
      float r = __int_as_float(0x7fc00000);
      if (row_ok && col < ep.P) r = corr_nan(tot[grp * 16 + e], rinv, ep.col_rmul[col]);
      const float a = (r == r) ? fabsf(r) : -1.0f;
      const unsigned b = __ballot_sync(0xffffffffu, ce >= 0.0f && a == ce);
      if (lane == e && b != 0u) {
        const long long marker = ep.marker_offset + row_base + (__ffs(b) - 1);
        atomicMax(ep.best + col, best_key(ce, marker));
      }
    }
  }
}

template <bool HAS_LO>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_scan(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
              const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
              int num_kb, int n_mt, int n_nt, int bn, const int* __restrict__ tflags,
              long long spin_ns, EpiParams ep) {
  // bn = B rows per tile: 256 for the phenotype panel, 64 for the covariate projection
  using C = Cfg<HAS_LO>;
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
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * C::kStageBytes + 8 * (2 * S + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  auto sA = [&](int s) { return base + s * C::kStageBytes; };
  auto sBhi = [&](int s) { return base + s * C::kStageBytes + A_BYTES; };
  auto sBlo = [&](int s) { return base + s * C::kStageBytes + A_BYTES + B_BYTES; };
  auto sAlo = [&](int s) { return base + s * C::kStageBytes + A_BYTES + 2 * B_BYTES; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
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
  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
    if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int stage = 0;
    uint32_t phase = 0;
    int armed[S];
#pragma unroll
    for (int s = 0; s < S; ++s) armed[s] = -1;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int mt, nt;
      tile_coord(tile, n_mt, n_nt, mt, nt);
      const bool lo = HAS_LO && tflags[mt] != 0;
      const uint32_t bytes = A_BYTES + 2u * (uint32_t)bn * (TBK * 2) + (lo ? A_BYTES : 0);
      for (int kb = 0; kb < num_kb; ++kb) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full_bar(stage), bytes);
        armed[stage] = (int)phase;
        tma_load_2d(&tmAhi, sA(stage), full_bar(stage), kb * TBK, mt * TBM);
        tma_load_2d(&tmBhi, sBhi(stage), full_bar(stage), kb * TBK, nt * bn);
        tma_load_2d(&tmBlo, sBlo(stage), full_bar(stage), kb * TBK, nt * bn);
        if (lo) tma_load_2d(&tmAlo, sAlo(stage), full_bar(stage), kb * TBK, mt * TBM);
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // copies still in flight land before the CTA leaves (bounded)
    for (int s = 0; s < S; ++s)
      if (armed[s] >= 0) mbar_wait(full_bar(s), (uint32_t)armed[s], abort_flag, spin_ns, ep.status);
    } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    // Each chunk of kChunkKB K blocks starts a fresh accumulator (no chained accumulation
    // across chunks); the two chunk accumulators alternate.
    int stage = 0;
    uint32_t phase = 0;
    uint32_t g = 0;
    bool ok = true;
    const uint32_t idesc = idesc_bf16(bn);
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int mt, nt;
      tile_coord(tile, n_mt, n_nt, mt, nt);
      const bool lo = HAS_LO && tflags[mt] != 0;
      for (int kb0 = 0; kb0 < num_kb && ok; kb0 += kChunkKB, ++g) {
        const int acc = (int)(g & 1u);
        const uint32_t ph = (g >> 1) & 1u;
        if (!mbar_wait(cempty_bar(acc), ph ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * TBN);
        const int kb1 = min(num_kb, kb0 + kChunkKB);
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, spin_ns, ep.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < TBK / 16; ++k) {
            const uint64_t a = sdesc_sw64(sA(stage) + 32u * k);
            const uint64_t bh = sdesc_sw64(sBhi(stage) + 32u * k);
            const uint64_t bl = sdesc_sw64(sBlo(stage) + 32u * k);
            tc_mma(d, a, bh, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
            tc_mma(d, a, bl, idesc, 1u);
            if (lo) tc_mma(d, sdesc_sw64(sAlo(stage) + 32u * k), bh, idesc, 1u);
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
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
    // ------------------------------------------------------------ epilogue
    // 8 warps: (TMEM lane quarter, column half) pairs; FP32 running totals in registers.
    const int quarter = warp & 3;
    const int half = (warp - 4) >> 2;
    uint32_t g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int mt, nt;
      tile_coord(tile, n_mt, n_nt, mt, nt);
      float tot[128];
#pragma unroll
      for (int e = 0; e < 128; ++e) tot[e] = 0.0f;
      for (int kb0 = 0; kb0 < num_kb; kb0 += kChunkKB, ++g) {
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
      const long long row_base = (long long)mt * TBM + quarter * 32;
      const long long row = row_base + lane;
      const bool row_ok = row < ep.M;
      const float rinv = (row_ok && ep.row_inv) ? ep.row_inv[row] : __int_as_float(0x7fc00000);
      if (ep.raw_out) {
        // covariate projection: the first raw_cols columns of the tile, unnormalised
        if (row_ok && half == 0) {
#pragma unroll
          for (int e = 0; e < 64; ++e)
            if (e < ep.raw_cols) ep.raw_out[row * ep.raw_ld + e] = tot[e];
        }
      } else {
        epilogue_tile(ep, tot, row, row_base, row_ok, rinv, nt * TBN + half * 128, lane);
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

template <bool HAS_LO>
cudaError_t go(const CUtensorMap* a, const CUtensorMap* alo, const CUtensorMap* bh,
               const CUtensorMap* bl, int64_t K, const int* tflags, const EpiParams& ep,
               int sm_count, long long spin_ns, cudaStream_t st) {
  using C = Cfg<HAS_LO>;
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_scan<HAS_LO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + TBM - 1) / TBM;
  const int bn = ep.raw_out ? 64 : TBN;
  const int n_nt = (ep.P + bn - 1) / bn;
  const int tiles = n_mt * n_nt;
  const int grid = tiles < sm_count ? tiles : sm_count;
  k_tc_scan<HAS_LO><<<grid, kThreads, C::kSmem, st>>>(*a, *alo, *bh, *bl, (int)(K / TBK), n_mt,
                                                       n_nt, bn, tflags, spin_ns, ep);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_scan(const CUtensorMap* tmAhi, const CUtensorMap* tmAlo,
                           const CUtensorMap* tmBhi, const CUtensorMap* tmBlo, int64_t K,
                           bool has_lo, const int* tflags, const EpiParams& ep, int sm_count,
                           long long spin_ns, cudaStream_t st) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  if (K % TBK) return cudaErrorInvalidValue;
  return has_lo ? go<true>(tmAhi, tmAlo, tmBhi, tmBlo, K, tflags, ep, sm_count, spin_ns, st)
                : go<false>(tmAhi, tmAhi, tmBhi, tmBlo, K, tflags, ep, sm_count, spin_ns, st);
}

cudaError_t launch_wait_test(const uint32_t* flag, long long limit_ns, uint32_t* result,
                             cudaStream_t st) {
  k_wait_test<<<1, 1, 0, st>>>(flag, limit_ns, result);
  return cudaGetLastError();
}

}  // namespace tg
