// The contraction of Eq. 2 (Section 2.2) on block-scaled FP4 tensor cores: an experimental
// low-precision multi-piece form for 2-bit calls (TG_PREC_FP4_PIECES).
//
// GB300 runs tcgen05.mma kind::mxf4 (E2M1 operands, an E8M0 scale per 32 elements) at several
// times the BF16 rate. Genotype counts {0, 1, 2} are exact in E2M1. The unit-norm panel is not,
// so each column v is scaled by a power of two 2^e that puts max |v| 2^e in (1.5, 3] and split
// into kFp4Pieces E2M1 pieces, piece k at scale 8^-k:
//   z = v 2^e ~= sum_k q_k 8^-k,  q_k = E2M1 nearest to (z - sum_{l<k} q_l 8^-l) 8^k.
// The residual before piece k, times 8^k, stays within [-4, 4] (the grid's gaps are at most 1 up
// to 4), so no piece saturates, and each piece cuts the residual by 8: six pieces leave it near
// 8^-5 / 2 of the column's scale, about the error of the BF16 hi + lo split (the accuracy is
// measured against the FP64 oracle in tests/test_gpu_fp4.py). The products of the pieces
// accumulate in one FP32 TMEM accumulator: each MMA carries piece k's scale 2^-3k as its B
// scale factor and 1 as A's, constants written once per CTA into tensor memory, so their TMEM
// layout and the descriptor's scale-factor ids do not matter.
// The statistics reuse the split form's epilogue: D = tot + shift * col_cs with shift = -mean
// (the centring add-back: col_cs = sum_i of the column's pieces) and r = D rinv rmul with
// rmul = 2^-e (the column's scale) or NaN for an untestable phenotype.
// Missing calls: the E2M1 operand cannot hold a marker's mean, so in this form a marker with a
// missing call has no test (NaN outputs; the marker norm kernel marks it).
#include <cuda.h>

#include "device.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace tg {
namespace {

using namespace tcx;

constexpr int kFBK = 128;           // samples per stage: 64 bytes of E2M1 per row
constexpr int kFChunkStages = 8;    // 1024 samples per accumulation chunk, as the split form
constexpr int kFThreads = 256;      // warp 0 producer, warp 1 MMA, warps 4..7 epilogue

// E2M1 magnitude codes 0..7 = {0, 0.5, 1, 1.5, 2, 3, 4, 6}; bit 3 is the sign.
__device__ __forceinline__ uint32_t e2m1_round(double t, double* q) {
  const double a = fabs(t);
  double m;
  uint32_t c;
  if (a < 1.75) {  // steps of 0.5 up to 1.5, and [1.75, 2) rounds to 2 below
    const double h = rint(a * 2.0);  // 0..3
    m = 0.5 * h;
    c = (uint32_t)h;
  } else if (a < 3.5) {  // 2 or 3
    m = a < 2.5 ? 2.0 : 3.0;
    c = a < 2.5 ? 4u : 5u;
  } else if (a < 5.0) {
    m = 4.0;
    c = 6u;
  } else {
    m = 6.0;
    c = 7u;
  }
  const bool neg = t < 0.0 && c != 0u;
  *q = neg ? -m : m;
  return c | (neg ? 8u : 0u);
}

// Pieces of one operand row (a panel column or a projection column) per block: out rows
// k * rows_pad + r for piece k, Npad / 2 bytes each (sample i in the low nibble of byte i / 2 when
// i is even); scale[r] = 2^-e, or NaN when the row is not a test (valid = 0, rows past the
// operand); cs[r] = sum over i and k of q_k 8^-k (the scaled column sum).
__global__ void __launch_bounds__(256) k_fp4_pieces(const double* __restrict__ src, long long lds,
                                                    const double* __restrict__ div,
                                                    const float* __restrict__ valid, int nrows,
                                                    int rows_pad, long long N, long long Npad,
                                                    uint8_t* __restrict__ out, float* __restrict__ scale,
                                                    float* __restrict__ cs) {
  __shared__ double red[33];
  const int r = blockIdx.x;
  const bool ok = r < nrows && (!valid || valid[r] == valid[r]);
  const double* v = src + (long long)r * lds;
  const double mul = (ok && div) ? 1.0 / div[r] : 1.0;
  double mx = 0.0;
  if (ok)
    for (long long i = threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, fabs(v[i] * mul));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    red[32] = m;
  }
  __syncthreads();
  mx = red[32];
  __syncthreads();
  const bool live = ok && mx > 0.0;
  const int e = live ? (int)floor(log2(3.0 / mx)) : 0;  // max |v| 2^e in (1.5, 3]
  const double up = ldexp(1.0, e);
  double sum = 0.0;
  const long long nbytes = Npad / 2;
  for (long long b = threadIdx.x; b < nbytes; b += blockDim.x) {
    uint32_t nib[kFp4Pieces][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long i = 2 * b + h;
      double res = (live && i < N) ? v[i] * mul * up : 0.0;
      double scale_k = 1.0;  // 8^-k
#pragma unroll
      for (int k = 0; k < kFp4Pieces; ++k) {
        double q;
        nib[k][h] = e2m1_round(res / scale_k, &q);
        res -= q * scale_k;
        sum += q * scale_k;
        scale_k *= 0.125;
      }
    }
#pragma unroll
    for (int k = 0; k < kFp4Pieces; ++k)
      out[((long long)k * rows_pad + r) * nbytes + b] = (uint8_t)(nib[k][0] | (nib[k][1] << 4));
  }
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) {
    scale[r] = live ? (float)ldexp(1.0, -e) : (ok ? 1.0f : __int_as_float(0x7fc00000));
    cs[r] = (float)sum;
  }
}

// Bit b of a 16-bit value to bit 2b.
__device__ __forceinline__ uint32_t spread2(uint32_t m) {
  m = (m | (m << 8)) & 0x00FF00FFu;
  m = (m | (m << 4)) & 0x0F0F0F0Fu;
  m = (m | (m << 2)) & 0x33333333u;
  m = (m | (m << 1)) & 0x55555555u;
  return m;
}
// Bits at the even positions 2b of a 32-bit value to bit b.
__device__ __forceinline__ uint32_t compact2(uint32_t m) {
  m &= 0x55555555u;
  m = (m | (m >> 1)) & 0x33333333u;
  m = (m | (m >> 2)) & 0x0F0F0F0Fu;
  m = (m | (m >> 4)) & 0x00FF00FFu;
  m = (m | (m >> 8)) & 0x0000FFFFu;
  return m;
}

// E2M1 codes of 16 2-bit fields (field 00, 2 copies -> 2.0 = code 4; 10 -> 1.0 = code 2; 11 and
// 01, missing -> 0), samples from `left` before N on (codes past N are 0): sample s's nibble at
// bits 4s of lo (s < 8) or of hi. Per field, code bit 2 is set for 00 and code bit 1 for 10;
// both flags move from bit 2s of the word to bit 4s of the output.
__device__ __forceinline__ uint2 e2m1_codes16(uint32_t w, int left) {
  if (left <= 0) return make_uint2(0u, 0u);
  const uint32_t a = w & 0x55555555u, b = (w >> 1) & 0x55555555u;
  const uint32_t two = compact2(~a & ~b);  // bit s: field s is 00
  const uint32_t one = compact2(~a & b);   // bit s: field s is 10
  uint32_t lo = (spread2(spread2(two & 0xFFu)) << 2) | (spread2(spread2(one & 0xFFu)) << 1);
  uint32_t hi = (spread2(spread2(two >> 8)) << 2) | (spread2(spread2(one >> 8)) << 1);
  if (left < 16) {
    const unsigned long long keep = (1ull << (4 * left)) - 1ull;
    lo &= (uint32_t)keep;
    hi &= (uint32_t)(keep >> 32);
  }
  return make_uint2(lo, hi);
}

// The FP4 form's decode of 2-bit rows in one pass, one warp per row: each lane takes 64-sample
// chunks (a 16-byte load of the packed row; G is 16-byte aligned, ldg a multiple of 16, and the
// chunk of a sample below N lies inside the row) and writes their E2M1 codes (32 bytes), and
// the warp sums the exact counts of the row (n_obs, S, S2, as the counting pass does) and writes
// n_obs, the FP64 mean S / n, |g_c|^2 = (n S2 - S^2) / n and shift = -mean (the epilogue's
// centring add-back; NaN mean and shift for a row without an observed call).
constexpr int kF4DecWarps = 8;
__global__ void __launch_bounds__(kF4DecWarps * 32) k_fp4_decode(
    const uint8_t* __restrict__ G, long long ldg, int N, long long M, uint8_t* __restrict__ A,
    long long lda, int32_t* __restrict__ nobs, double* __restrict__ mean_out,
    double* __restrict__ gc2_out, float* __restrict__ shift) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * kF4DecWarps + warp;
  if (j >= M) return;
  const uint4* row = reinterpret_cast<const uint4*>(G + j * ldg);
  uint4* out = reinterpret_cast<uint4*>(A + j * lda);
  const int chunks = (int)(lda / 32);  // 64 samples each: 32 bytes of codes
  unsigned long long n = 0, S = 0, S2 = 0;
  for (int c = lane; c < chunks; c += 32) {
    const int i0 = c * 64;
    uint2 q[4] = {make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u)};
    if (i0 < N) {
      const uint4 v = __ldg(row + c);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        q[k] = e2m1_codes16(w4[k], N - (i0 + 16 * k));
        count16_2bit(w4[k], N - (i0 + 16 * k), n, S, S2);
      }
    }
    out[2 * c] = make_uint4(q[0].x, q[0].y, q[1].x, q[1].y);
    out[2 * c + 1] = make_uint4(q[2].x, q[2].y, q[3].x, q[3].y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    S += __shfl_xor_sync(0xffffffffu, S, o);
    S2 += __shfl_xor_sync(0xffffffffu, S2, o);
  }
  if (lane == 0) {
    const double dn = (double)n;
    const double mean = n ? (double)S / dn : __longlong_as_double(0x7ff8000000000000ll);
    const long long num = (long long)S2 * (long long)n - (long long)S * (long long)S;
    nobs[j] = (int32_t)n;
    mean_out[j] = mean;
    gc2_out[j] = n ? (double)num / dn : __longlong_as_double(0x7ff8000000000000ll);
    shift[j] = -(float)mean;
  }
}

__device__ __forceinline__ void tc_mma_fp4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], "
      "p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::mxf4 with block scaling: A and B E2M1 (format code 1 in bits
// 7-9 and 10-12), both K-major, N >> 3 in bits 17-22, E8M0 scale factors (bit 23), M >> 4 in
// bits 24-28; scale-factor ids 0 (the scale factors are constants, so any id reads the same).
__host__ __device__ constexpr uint32_t idesc_mxf4(int m, int n) {
  return (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (1u << 23) |
         ((uint32_t)(m >> 4) << 24);
}

template <int BN>
struct F4Cfg {
  static constexpr int kABytes = TBM * 64;               // 128 rows x 128 samples
  static constexpr int kBBytes = BN * 64;                // one piece
  static constexpr int kStageBytes = kABytes + kFp4Pieces * kBBytes;
  static constexpr int kStages = BN == 128 ? 3 : 5;
  static constexpr int kSmem = kStages * kStageBytes + 256 + 1024;
  static constexpr int kSfCol = 256;                     // TMEM: A's scale, then each piece's
  static_assert(2 * BN <= kSfCol && kSfCol + 4 * (1 + kFp4Pieces) <= kTmemCols, "TMEM");
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

// Persistent, one CTA per SM: tiles of 128 markers x BN columns (BN = 128: the panel, with the
// statistics epilogue; BN = 64: the covariate projection, raw). Warp 0 lane 0 loads each stage's
// A (128 rows x 64 bytes) and kFp4Pieces B boxes (BN rows x 64 bytes) by TMA (64-byte swizzle);
// warp 1 lane 0 issues 2 K-steps x kFp4Pieces block-scaled MMAs per stage into a chunk
// accumulator; warps 4..7 (one TMEM lane quarter each, one marker row per thread) write the
// scale-factor constants once, drain each chunk into FP32 totals and run the epilogue.
template <int BN>
__global__ void __launch_bounds__(kFThreads, 1)
    k_fp4_scan(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int b_rows_pad, int num_st, int n_mt, int n_nt, int group_m, long long spin_ns,
               EpiParams ep) {
  using C = F4Cfg<BN>;
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
  auto sA = [&](int s) { return base + (uint32_t)(s * C::kStageBytes); };
  auto sB = [&](int s, int k) {
    return base + (uint32_t)(s * C::kStageBytes + C::kABytes + k * C::kBBytes);
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(cfull_bar(a), 1);
      mbar_init(cempty_bar(a), 4);
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
  if (warp >= 4) {  // the scale factors: 1 for A, 2^-3k for piece k (E8M0 127 - 3k), every byte
    const uint32_t la = (uint32_t)((warp - 4) * 32) << 16;
    for (int k = 0; k <= kFp4Pieces; ++k) {
      const uint32_t e8 = k == 0 ? 127u : 127u - 3u * (uint32_t)(k - 1);
      const uint32_t v = e8 * 0x01010101u;
      asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(
                       tmem_base + la + (uint32_t)(C::kSfCol + 4 * k)),
                   "r"(v)
                   : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const int num_tiles = n_mt * n_nt;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int mt, nt;
      tile_coord(tile, n_mt, n_nt, group_m, mt, nt);
      for (int st = 0; st < num_st; ++st) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full_bar(stage), (uint32_t)C::kStageBytes);
        tma_load_2d(&tmA, sA(stage), full_bar(stage), st * 64, mt * TBM);
#pragma unroll
        for (int k = 0; k < kFp4Pieces; ++k)
          tma_load_2d(&tmB, sB(stage, k), full_bar(stage), st * 64, k * b_rows_pad + nt * BN);
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    for (int s = 0; s < S; ++s)  // copies in flight land before the CTA leaves (bounded)
      mbar_wait(full_bar(s), phase ^ (s < stage ? 0u : 1u), abort_flag, spin_ns, ep.status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_mxf4(TBM, BN);
    const uint32_t sfa = tmem_base + (uint32_t)C::kSfCol;
    int stage = 0;
    uint32_t phase = 0, g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      for (int st0 = 0; st0 < num_st && ok; st0 += kFChunkStages, ++g) {
        const int acc = (int)(g & 1u);
        if (!mbar_wait(cempty_bar(acc), ((g >> 1) & 1u) ^ 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * BN);
        const int st1 = min(num_st, st0 + kFChunkStages);
        for (int st = st0; st < st1; ++st) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, spin_ns, ep.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {  // two K-steps of 64 samples (32 bytes per row)
            const uint64_t a = sdesc_sw64(sA(stage) + 32u * kk);
#pragma unroll
            for (int k = 0; k < kFp4Pieces; ++k)
              tc_mma_fp4(d, a, sdesc_sw64(sB(stage, k) + 32u * kk), idesc, sfa,
                         sfa + 4u * (uint32_t)(k + 1), (st > st0 || kk > 0 || k > 0) ? 1u : 0u);
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
    tc_commit(drain_bar);
    mbar_wait(drain_bar, 0u, abort_flag, spin_ns, ep.status);
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp - 4;
    const uint32_t la = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int mt, nt;
      tile_coord(tile, n_mt, n_nt, group_m, mt, nt);
      float tot[BN];
#pragma unroll
      for (int e = 0; e < BN; ++e) tot[e] = 0.0f;
      for (int st0 = 0; st0 < num_st; st0 += kFChunkStages, ++g) {
        const int acc = (int)(g & 1u);
        if (!mbar_wait(cfull_bar(acc), (g >> 1) & 1u, abort_flag, spin_ns, ep.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int i = 0; i < BN / 32; ++i) {
          float v[32];
          __syncwarp();
          tc_ld32(tmem_base + la + (uint32_t)(acc * BN + i * 32), v);
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
      const float shift = (row_ok && ep.row_shift) ? ep.row_shift[row] : 0.0f;
      if (BN == 64) {  // the projection: raw products with the add-back, in column units
        if (row_ok) {
#pragma unroll
          for (int e = 0; e < BN; ++e)
            if (e < ep.raw_cols)
              ep.raw_out[row * ep.raw_ld + e] = fmaf(shift, ep.col_cs[e], tot[e]) * ep.col_rmul[e];
        }
      } else {
        const float rinv = (row_ok && ep.row_inv) ? ep.row_inv[row] : __int_as_float(0x7fc00000);
        epilogue_tile(ep, *reinterpret_cast<float(*)[128]>(tot), row, row_base, row_ok, rinv, shift,
                      nt * BN, lane);
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

template <int BN>
cudaError_t go_fp4(const CUtensorMap* a, const CUtensorMap* b, int b_rows_pad, int64_t Npad,
                   const EpiParams& ep, int sm_count, long long spin_ns, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_fp4_scan<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         F4Cfg<BN>::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_mt = (ep.M + TBM - 1) / TBM;
  const int n_nt = (ep.P + BN - 1) / BN;
  const int tiles = n_mt * n_nt;
  const int grid = tiles < sm_count ? tiles : sm_count;
  const int num_st = (int)((Npad + kFBK - 1) / kFBK);
  k_fp4_scan<BN><<<grid, kFThreads, F4Cfg<BN>::kSmem, st>>>(*a, *b, b_rows_pad, num_st, n_mt, n_nt,
                                                            16, spin_ns, ep);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp4_pieces(const double* src, int64_t lds, const double* div, const float* valid,
                              int64_t nrows, int64_t rows_pad, int64_t N, int64_t Npad, uint8_t* out,
                              float* scale, float* cs, cudaStream_t st) {
  if (rows_pad <= 0) return cudaSuccess;
  k_fp4_pieces<<<(unsigned)rows_pad, 256, 0, st>>>(src, lds, div, valid, (int)nrows, (int)rows_pad,
                                                   N, Npad, out, scale, cs);
  return cudaGetLastError();
}

cudaError_t launch_fp4_decode(const uint8_t* G, int64_t ldg, int64_t N, int64_t M, uint8_t* A,
                              int64_t lda, int32_t* nobs, double* mean, double* gc2, float* shift,
                              cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  if (lda % 32 || ldg % 16 || lda * 2 < N) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((M + kF4DecWarps - 1) / kF4DecWarps);
  k_fp4_decode<<<grid, kF4DecWarps * 32, 0, st>>>(G, ldg, (int)N, M, A, lda, nobs, mean, gc2,
                                                   shift);
  return cudaGetLastError();
}

cudaError_t launch_fp4_scan(const CUtensorMap* tmA, const CUtensorMap* tmB, int b_rows_pad,
                            int64_t Npad, const EpiParams& ep, int sm_count, long long spin_ns,
                            cudaStream_t st) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  if (ep.raw_out) {
    if (ep.P > 64 || ep.raw_cols != ep.P) return cudaErrorInvalidValue;
    return go_fp4<64>(tmA, tmB, b_rows_pad, Npad, ep, sm_count, spin_ns, st);
  }
  return go_fp4<128>(tmA, tmB, b_rows_pad, Npad, ep, sm_count, spin_ns, st);
}

}  // namespace tg
