// Genotype decode with mean imputation (Section 2.2: genotypes processed in batches of markers).
//
// One warp per marker row. Pass 1 reads the packed row with 16-byte loads and counts,
// exactly in integers, the observed calls n, their sum S and sum of squares S2 (decode
// units: allele-1 counts for 2-bit calls, bytes for dosages); mean = S / n is one IEEE
// division and |g_c|^2 = (n S2 - S^2) / n one more. Pass 2 re-reads the row (cache-hot)
// and writes the contraction operand with 16-byte stores, zero past N:
//   FP32 form: the code of an observed call, the mean at a missing one.
//   split form (bf16): the row shifted by c = the mean rounded to a grid on which every
//   observed value minus c is exact in bf16 (2-bit: multiples of 2^-7, |code - c| <= 2;
//   dosage: integers, |byte - c| <= 255), and bf16(mean - c) at a missing call
//   (|mean - c| <= 2^-8 or 1/2, so its rounding error is <= 2^-17 or 2^-10). The scan adds
//   c * sum_i y_i back per phenotype column, so imputation needs no extra product.
//
// 2-bit fields follow the PLINK 1 .bed table: 00 -> 2, 10 -> 1, 11 -> 0, 01 -> missing.
// With lo = w & 0x55.. and hi = (w >> 1) & 0x55.. per 32-bit word: count 2 = ~lo & ~hi,
// count 1 = hi & ~lo, count 0 = lo & hi, missing = lo & ~hi.
//
// The split writer takes 16 samples per lane and step (one packed word of 2-bit fields, or
// 16 dosage bytes) and stores 32 bytes:
//   2-bit: the row's four possible bf16 values, indexed by the raw field, sit in two words;
//     one byte permute per pair of fields picks both values.
//   dosage: a byte permute builds the float 2^23 + b, and subtracting 2^23 + c leaves b - c
//     exactly; pairs are rounded to bf16x2 in one conversion.
#include <cuda_bf16.h>

#include "device.cuh"
#include "genotype.cuh"
#include "internal.h"

namespace tg {
namespace {

constexpr int kWarps = 8;
constexpr int kWarpRowN = 4096;  // split-form rows up to this many samples: one warp per row

template <int ENC>
__device__ __forceinline__ void row_stats(const uint8_t* __restrict__ row, int N,
                                          const uint32_t* __restrict__ mrow, int lane,
                                          unsigned long long& n, unsigned long long& S,
                                          unsigned long long& S2) {
  n = S = S2 = 0;
  if (ENC == TG_ENC_2BIT) {
    const int nb = (N + 3) >> 2;
    const int nchunk = (nb + 15) >> 4;
#pragma unroll 4
    for (int c = lane; c < nchunk; c += 32) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + c);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)  // word q: samples from c * 64 + q * 16
        count16_2bit(w4[q], N - (c * 64 + q * 16), n, S, S2);
    }
  } else {
    const int nchunk = (N + 15) >> 4;
#pragma unroll 4
    for (int c = lane; c < nchunk; c += 32) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + c);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
      uint32_t skip = 0;  // bit k: byte k of the chunk is missing or past N
      if (mrow) skip = (mrow[(c * 16) >> 5] >> ((c * 16) & 31)) & 0xFFFFu;
      const int left = N - c * 16;
      if (left < 16) skip |= 0xFFFFu << left;
      if (skip == 0) {  // 16 observed bytes: sums of bytes and of their squares by dp4a
        uint32_t s1 = 0, s2 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          s1 = __dp4a(w4[q], 0x01010101u, s1);
          s2 = __dp4a(w4[q], w4[q], s2);
        }
        n += 16;
        S += s1;
        S2 += s2;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t u = (w4[q] >> (8 * b)) & 0xFFu;
            if (!((skip >> (q * 4 + b)) & 1u)) {
              n += 1;
              S += u;
              S2 += u * u;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    S += __shfl_xor_sync(0xffffffffu, S, o);
    S2 += __shfl_xor_sync(0xffffffffu, S2, o);
  }
}

// 8 decoded samples starting at i0 (a multiple of 8): values and missing bits.
template <int ENC>
__device__ __forceinline__ void load8(const uint8_t* __restrict__ row, const uint32_t* __restrict__ mrow,
                                      int i0, int N, float v[8], uint32_t& miss) {
  miss = 0;
  if (ENC == TG_ENC_2BIT) {
    const uint32_t w = *reinterpret_cast<const uint16_t*>(row + (i0 >> 2));
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t f = (w >> (2 * s)) & 3u;
      v[s] = (f == 0u) ? 2.0f : (f == 2u) ? 1.0f : 0.0f;
      if (f == 1u && i0 + s < N) miss |= 1u << s;
    }
  } else {
    const uint2 w = *reinterpret_cast<const uint2*>(row + i0);
    if (mrow) miss = (mrow[i0 >> 5] >> (i0 & 31)) & 0xFFu;
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = (float)(((s < 4 ? w.x : w.y) >> (8 * (s & 3))) & 0xFFu);
  }
#pragma unroll
  for (int s = 0; s < 8; ++s)
    if (i0 + s >= N) v[s] = 0.0f;
  if (i0 + 8 > N) miss &= (N > i0) ? ((1u << (N - i0)) - 1u) : 0u;
}

// Shift of a marker row for the split form (see above); 0 when no call is observed.
template <int ENC>
__device__ __forceinline__ double row_shift(unsigned long long n, double mean) {
  if (!n) return 0.0;
  return ENC == TG_ENC_2BIT ? rint(mean * 128.0) * (1.0 / 128.0) : rint(mean);
}

template <int ENC, int PREC>
__global__ void __launch_bounds__(kWarps * 32) k_decode(
    const uint8_t* __restrict__ G, long long ldg, int N, long long M,
    const uint32_t* __restrict__ miss, long long ldm, void* __restrict__ Ahi,
    float* __restrict__ shift_out, uint32_t* __restrict__ mh_out, long long lda,
    int32_t* __restrict__ nobs_out, long long* __restrict__ S_out, long long* __restrict__ S2_out,
    double* __restrict__ mean_out, double* __restrict__ gc2_out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * kWarps + warp;
  if (j >= M) return;
  const uint8_t* row = G + j * ldg;
  const uint32_t* mrow = miss ? miss + j * ldm : nullptr;
  unsigned long long n, S, S2;
  row_stats<ENC>(row, N, mrow, lane, n, S, S2);
  const double dn = (double)n;
  const double mean = n ? (double)S / dn : __longlong_as_double(0x7ff8000000000000ll);
  if (lane == 0) {
    if (nobs_out) nobs_out[j] = (int32_t)n;
    if (S_out) S_out[j] = (long long)S;
    if (S2_out) S2_out[j] = (long long)S2;
    if (mean_out) mean_out[j] = mean;
    if (gc2_out) {
      const long long num = (long long)S2 * (long long)n - (long long)S * (long long)S;
      gc2_out[j] = n ? (double)num / dn : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
  // pass 2: operand row (skipped when Ahi is NULL: the statistics and the split form's
  // per-row shift and missing value only, for the contraction that decodes in its producer)
  const double m_imp = n ? mean : 0.0;
  const long long steps = lda >> 3;
  if (PREC == TG_PREC_SPLIT_BF16) {
    const double c = row_shift<ENC>(n, mean);
    const float cf = (float)c;  // exact: a multiple of 2^-7 in [0, 2] or an integer in [0, 255]
    const __nv_bfloat16 mh = __double2bfloat16(m_imp - c);
    const uint32_t mhu = (uint32_t)__bfloat16_as_ushort(mh);
    if (lane == 0 && shift_out) shift_out[j] = cf;
    if (lane == 0 && mh_out) mh_out[j] = mhu;
    if (!Ahi) return;
    uint4* ah = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(Ahi) + j * lda);
    const long long groups = lda >> 4;  // 16 samples each
    if (ENC == TG_ENC_2BIT) {
      auto bits = [](float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); };
      const uint32_t lut0 = bits(2.0f - cf) | (mhu << 16);
      const uint32_t lut1 = bits(1.0f - cf) | (bits(-cf) << 16);
      const uint32_t* wrow = reinterpret_cast<const uint32_t*>(row);
#pragma unroll 2
      for (long long t = lane; t < groups; t += 32) {
        const int i0 = (int)(t << 4);
        uint32_t o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (i0 < N) {
          split16_2bit(__ldg(wrow + t), lut0, lut1, o);
          if (i0 + 16 > N) zero_tail16(o, i0, N);
        }
        ah[2 * t] = make_uint4(o[0], o[1], o[2], o[3]);
        ah[2 * t + 1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
    } else {
      const float c_plus = 8388608.0f + cf;  // 2^23 + c, exact
      const uint32_t mh2 = mhu | (mhu << 16);
      const uint4* vrow = reinterpret_cast<const uint4*>(row);
#pragma unroll 2
      for (long long t = lane; t < groups; t += 32) {
        const int i0 = (int)(t << 4);
        uint32_t o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (i0 < N) {
          const uint32_t ms = mrow ? (mrow[i0 >> 5] >> (i0 & 31)) & 0xFFFFu : 0u;
          split16_u8(__ldg(vrow + t), c_plus, ms, mh2, o);
          if (i0 + 16 > N) zero_tail16(o, i0, N);
        }
        ah[2 * t] = make_uint4(o[0], o[1], o[2], o[3]);
        ah[2 * t + 1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
    }
  } else {
    const float mf = (float)m_imp;
    float* af = reinterpret_cast<float*>(Ahi) + j * lda;
#pragma unroll 4
    for (long long t = lane; t < steps; t += 32) {
      const int i0 = (int)(t << 3);
      float v[8];
      uint32_t ms = 0;
      if (i0 < N) {
        load8<ENC>(row, mrow, i0, N, v, ms);
      } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = 0.0f;
      }
#pragma unroll
      for (int s = 0; s < 8; ++s)
        if ((ms >> s) & 1u) v[s] = mf;
      reinterpret_cast<float4*>(af + i0)[0] = make_float4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<float4*>(af + i0)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
}

// Split form for rows of up to THREADS * GPT * 16 samples: one block per marker row, the
// packed row held in registers between the two passes (one read of the row from HBM, every
// load of a thread in flight at once). Used for dosage rows, where the warp-per-row kernel's
// second read of a 23 KB row misses L2 under load.

template <int ENC, int GPT, int THREADS>
__global__ void __launch_bounds__(THREADS, GPT * THREADS <= 1536 ? 4 : 2) k_decode_rows(
    const uint8_t* __restrict__ G, long long ldg, int N, const uint32_t* __restrict__ miss,
    long long ldm, __nv_bfloat16* __restrict__ A, float* __restrict__ shift_out,
    uint32_t* __restrict__ mh_out, long long lda, int32_t* __restrict__ nobs_out,
    long long* __restrict__ S_out, long long* __restrict__ S2_out, double* __restrict__ mean_out,
    double* __restrict__ gc2_out) {
  __shared__ unsigned long long red[3][THREADS / 32];
  __shared__ float s_c;
  __shared__ uint32_t s_mh;
  const long long j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint8_t* row = G + j * ldg;
  const uint32_t* mrow = miss ? miss + j * ldm : nullptr;
  const int nvalid = (N + 15) >> 4;  // 16-sample groups holding a sample < N
  // pass 1: load this thread's groups, count n, S, S2
  uint32_t w[GPT];  // 2-bit: one word of 16 fields per group
  uint4 v[GPT];     // dosage: 16 bytes per group
  uint32_t ms[GPT]; // dosage: missing bits of the group
  uint32_t n = 0, S = 0, S2 = 0;
#pragma unroll
  for (int g = 0; g < GPT; ++g) {
    const int t = tid + g * THREADS;
    if (ENC == TG_ENC_2BIT) {
      w[g] = t < nvalid ? __ldg(reinterpret_cast<const uint32_t*>(row) + t) : 0u;
    } else {
      v[g] = t < nvalid ? __ldg(reinterpret_cast<const uint4*>(row) + t) : make_uint4(0, 0, 0, 0);
      ms[g] = (t < nvalid && mrow) ? (mrow[t >> 1] >> ((t & 1) * 16)) & 0xFFFFu : 0u;
    }
  }
#pragma unroll
  for (int g = 0; g < GPT; ++g) {
    const int t = tid + g * THREADS;
    if (t >= nvalid) continue;
    const int left = N - t * 16;  // >= 1
    if (ENC == TG_ENC_2BIT) {
      const uint32_t valid = left >= 16 ? 0x55555555u : (0x55555555u & ((1u << (2 * left)) - 1u));
      const uint32_t lo = w[g] & 0x55555555u, hi = (w[g] >> 1) & 0x55555555u;
      const uint32_t two = ~lo & ~hi & valid, one = hi & ~lo & valid, zero = lo & hi & valid;
      const uint32_t c2 = __popc(two), c1 = __popc(one);
      n += c2 + c1 + __popc(zero);
      S += 2 * c2 + c1;
      S2 += 4 * c2 + c1;
    } else {
      uint32_t skip = ms[g];
      if (left < 16) skip |= 0xFFFFu << left;
      const uint32_t w4[4] = {v[g].x, v[g].y, v[g].z, v[g].w};
      if (skip == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          S = __dp4a(w4[q], 0x01010101u, S);
          S2 = __dp4a(w4[q], w4[q], S2);
        }
        n += 16;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t u = (w4[q] >> (8 * b)) & 0xFFu;
            if (!((skip >> (q * 4 + b)) & 1u)) {
              n += 1;
              S += u;
              S2 += u * u;
            }
          }
      }
    }
  }
  unsigned long long n64 = n, S64 = S, S264 = S2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    S64 += __shfl_xor_sync(0xffffffffu, S64, o);
    S264 += __shfl_xor_sync(0xffffffffu, S264, o);
  }
  if (lane == 0) {
    red[0][warp] = n64;
    red[1][warp] = S64;
    red[2][warp] = S264;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long tn = 0, tS = 0, tS2 = 0;
#pragma unroll
    for (int k = 0; k < THREADS / 32; ++k) {
      tn += red[0][k];
      tS += red[1][k];
      tS2 += red[2][k];
    }
    const double dn = (double)tn;
    const double mean = tn ? (double)tS / dn : __longlong_as_double(0x7ff8000000000000ll);
    if (nobs_out) nobs_out[j] = (int32_t)tn;
    if (S_out) S_out[j] = (long long)tS;
    if (S2_out) S2_out[j] = (long long)tS2;
    if (mean_out) mean_out[j] = mean;
    if (gc2_out) {
      const long long num = (long long)tS2 * (long long)tn - (long long)tS * (long long)tS;
      gc2_out[j] = tn ? (double)num / dn : __longlong_as_double(0x7ff8000000000000ll);
    }
    const double c = row_shift<ENC>(tn, mean);
    if (shift_out) shift_out[j] = (float)c;
    s_c = (float)c;
    s_mh = (uint32_t)__bfloat16_as_ushort(__double2bfloat16((tn ? mean : 0.0) - c));
    if (mh_out) mh_out[j] = s_mh;
  }
  // without an operand (the contraction decodes in its producer): the statistics, the shift
  // and the missing value only
  if (!A) return;
  __syncthreads();
  // pass 2: the operand row from registers, zeros past N
  const float cf = s_c;
  const uint32_t mhu = s_mh;
  uint4* ah = reinterpret_cast<uint4*>(A + j * lda);
  auto bits = [](float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); };
  const uint32_t lut0 = bits(2.0f - cf) | (mhu << 16);
  const uint32_t lut1 = bits(1.0f - cf) | (bits(-cf) << 16);
  const float c_plus = 8388608.0f + cf;
  const uint32_t mh2 = mhu | (mhu << 16);
#pragma unroll
  for (int g = 0; g < GPT; ++g) {
    const int t = tid + g * THREADS;
    if (t >= nvalid) break;
    uint32_t o[8];
    if (ENC == TG_ENC_2BIT)
      split16_2bit(w[g], lut0, lut1, o);
    else
      split16_u8(v[g], c_plus, ms[g], mh2, o);
    if (t * 16 + 16 > N) zero_tail16(o, t * 16, N);
    ah[2 * t] = make_uint4(o[0], o[1], o[2], o[3]);
    ah[2 * t + 1] = make_uint4(o[4], o[5], o[6], o[7]);
  }
  const long long groups = lda >> 4;
  for (long long t = nvalid + tid; t < groups; t += THREADS) {
    ah[2 * t] = make_uint4(0, 0, 0, 0);
    ah[2 * t + 1] = make_uint4(0, 0, 0, 0);
  }
}

// |g_c|^2 of each marker over the samples of a subset panel, in decode units, the marker's
// missing calls imputed with its all-sample mean m (one warp per marker). With n observed
// calls in the subset (sum T, sum of squares U, exact integers), k imputed ones and N_S = n + k,
// the subset mean is gbar = (T + k m) / N_S and
//   |g_c|^2 = (n U - T^2) / n + n (T / n - gbar)^2 + k (m - gbar)^2,
// the first term exact in integers, the others small and well conditioned.
__device__ __forceinline__ uint32_t spread16(uint32_t m) {  // bit b -> bit 2b
  m = (m | (m << 8)) & 0x00FF00FFu;
  m = (m | (m << 4)) & 0x0F0F0F0Fu;
  m = (m | (m << 2)) & 0x33333333u;
  m = (m | (m << 1)) & 0x55555555u;
  return m;
}

template <int ENC>
__global__ void __launch_bounds__(kWarps * 32) k_subset_stats(
    const uint8_t* __restrict__ G, long long ldg, int N, long long M,
    const uint32_t* __restrict__ miss, long long ldm, const uint32_t* __restrict__ samples,
    const double* __restrict__ mean, double* __restrict__ gc2s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * kWarps + warp;
  if (j >= M) return;
  const uint8_t* row = G + j * ldg;
  const uint32_t* mrow = miss ? miss + j * ldm : nullptr;
  unsigned long long n = 0, T = 0, U = 0, k = 0;
  const int groups = (N + 15) >> 4;  // 16 samples each
  for (int t = lane; t < groups; t += 32) {
    const int left = N - t * 16;
    const uint32_t in_n = left >= 16 ? 0xFFFFu : ((1u << left) - 1u);
    const uint32_t s16 = (samples[t >> 1] >> ((t & 1) * 16)) & in_n;
    if (!s16) continue;
    if (ENC == TG_ENC_2BIT) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(row) + t);
      const uint32_t sm = spread16(s16);
      const uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;
      const uint32_t c2 = __popc(~lo & ~hi & sm), c1 = __popc(hi & ~lo & sm);
      n += c2 + c1 + __popc(lo & hi & sm);
      T += 2 * c2 + c1;
      U += 4 * c2 + c1;
      k += __popc(lo & ~hi & sm);
    } else {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + t);
      const uint32_t m16 = mrow ? (mrow[t >> 1] >> ((t & 1) * 16)) & 0xFFFFu : 0u;
      const uint32_t use = s16 & ~m16;
      k += __popc(s16 & m16);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if ((use >> (q * 4 + b)) & 1u) {
            const uint32_t u = (w4[q] >> (8 * b)) & 0xFFu;
            n += 1;
            T += u;
            U += u * u;
          }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    T += __shfl_xor_sync(0xffffffffu, T, o);
    U += __shfl_xor_sync(0xffffffffu, U, o);
    k += __shfl_xor_sync(0xffffffffu, k, o);
  }
  if (lane) return;
  if (n == 0) {  // every call of the subset imputed: constant there
    gc2s[j] = 0.0;
    return;
  }
  const double m = mean[j], dn = (double)n, dk = (double)k;
  const double gbar = ((double)T + dk * m) / (dn + dk);
  const long long num = (long long)U * (long long)n - (long long)T * (long long)T;
  const double d1 = (double)T / dn - gbar, d2 = m - gbar;
  gc2s[j] = (double)num / dn + dn * d1 * d1 + (k ? dk * d2 * d2 : 0.0);
}

template <int ENC, int PREC>
cudaError_t go(const uint8_t* G, int64_t ldg, int64_t N, int64_t M, const uint32_t* missing,
               int64_t ldm, void* Ahi, float* shift, uint32_t* mh, int64_t lda, int32_t* nobs,
               int64_t* S, int64_t* S2, double* mean, double* gc2, cudaStream_t st) {
  // Split form: one block per marker row with the row in registers (read from HBM once):
  // 256 threads x 6 groups of 16 samples for dosage rows, 128 x 12 for 2-bit rows; 12 and 24
  // groups up to twice those N, with or without the operand (Ahi NULL: statistics, shift and
  // missing value only). Short rows (N <= kWarpRowN: at most 8 groups per lane) and long ones
  // go to the warp-per-row kernel: a block per short row would leave most of its threads idle
  // and take several waves of blocks for a block of short rows.
  if constexpr (PREC == TG_PREC_SPLIT_BF16) {
    if (N <= kWarpRowN) {
      const unsigned grid = (unsigned)((M + kWarps - 1) / kWarps);
      k_decode<ENC, PREC><<<grid, kWarps * 32, 0, st>>>(
          G, ldg, (int)N, M, missing, ldm, Ahi, shift, mh, lda, nobs,
          reinterpret_cast<long long*>(S), reinterpret_cast<long long*>(S2), mean, gc2);
      return cudaGetLastError();
    }
    constexpr int T = ENC == TG_ENC_2BIT ? 128 : 256;
    constexpr int G1 = ENC == TG_ENC_2BIT ? 12 : 6;
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(Ahi);
    long long* S64 = reinterpret_cast<long long*>(S);
    long long* S264 = reinterpret_cast<long long*>(S2);
    if (N <= T * G1 * 16) {
      k_decode_rows<ENC, G1, T><<<(unsigned)M, T, 0, st>>>(G, ldg, (int)N, missing, ldm, A, shift,
                                                          mh, lda, nobs, S64, S264, mean, gc2);
      return cudaGetLastError();
    }
    if (N <= T * 2 * G1 * 16) {
      k_decode_rows<ENC, 2 * G1, T><<<(unsigned)M, T, 0, st>>>(G, ldg, (int)N, missing, ldm, A,
                                                              shift, mh, lda, nobs, S64, S264,
                                                              mean, gc2);
      return cudaGetLastError();
    }
  }
  const unsigned grid = (unsigned)((M + kWarps - 1) / kWarps);
  k_decode<ENC, PREC><<<grid, kWarps * 32, 0, st>>>(
      G, ldg, (int)N, M, missing, ldm, Ahi, shift, mh, lda, nobs, reinterpret_cast<long long*>(S),
      reinterpret_cast<long long*>(S2), mean, gc2);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decode(const uint8_t* G, int64_t ldg, int encoding, int64_t N, int64_t M,
                          const uint32_t* missing, int64_t ldm, int precision, void* Ahi,
                          float* shift, uint32_t* mh, int64_t lda, int32_t* nobs, int64_t* S,
                          int64_t* S2, double* mean, double* gc2, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  if (!Ahi && precision != TG_PREC_SPLIT_BF16) return cudaErrorInvalidValue;
  if (encoding == TG_ENC_2BIT) {
    return precision == TG_PREC_SPLIT_BF16
               ? go<TG_ENC_2BIT, TG_PREC_SPLIT_BF16>(G, ldg, N, M, missing, ldm, Ahi, shift, mh, lda, nobs, S, S2, mean, gc2, st)
               : go<TG_ENC_2BIT, TG_PREC_FP32>(G, ldg, N, M, missing, ldm, Ahi, shift, mh, lda, nobs, S, S2, mean, gc2, st);
  }
  return precision == TG_PREC_SPLIT_BF16
             ? go<TG_ENC_U8_DOSAGE, TG_PREC_SPLIT_BF16>(G, ldg, N, M, missing, ldm, Ahi, shift, mh, lda, nobs, S, S2, mean, gc2, st)
             : go<TG_ENC_U8_DOSAGE, TG_PREC_FP32>(G, ldg, N, M, missing, ldm, Ahi, shift, mh, lda, nobs, S, S2, mean, gc2, st);
}

cudaError_t launch_subset_stats(const uint8_t* G, int64_t ldg, int encoding, int64_t N, int64_t M,
                                const uint32_t* missing, int64_t ldm, const uint32_t* samples,
                                const double* mean, double* gc2s, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((M + kWarps - 1) / kWarps);
  if (encoding == TG_ENC_2BIT)
    k_subset_stats<TG_ENC_2BIT><<<grid, kWarps * 32, 0, st>>>(G, ldg, (int)N, M, missing, ldm,
                                                               samples, mean, gc2s);
  else
    k_subset_stats<TG_ENC_U8_DOSAGE><<<grid, kWarps * 32, 0, st>>>(G, ldg, (int)N, M, missing, ldm,
                                                                    samples, mean, gc2s);
  return cudaGetLastError();
}

}  // namespace tg
