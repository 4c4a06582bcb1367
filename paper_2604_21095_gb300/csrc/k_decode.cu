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
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

constexpr int kWarps = 8;

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
      for (int q = 0; q < 4; ++q) {
        const int base = c * 64 + q * 16;  // first sample of this word
        const int left = N - base;
        if (left <= 0) break;
        const uint32_t valid =
            (left >= 16) ? 0x55555555u : (0x55555555u & ((1u << (2 * left)) - 1u));
        const uint32_t w = w4[q];
        const uint32_t lo = w & 0x55555555u;
        const uint32_t hi = (w >> 1) & 0x55555555u;
        const uint32_t two = ~lo & ~hi & valid;
        const uint32_t one = hi & ~lo & valid;
        const uint32_t zero = lo & hi & valid;
        const int c2 = __popc(two), c1 = __popc(one);
        n += (unsigned)(c2 + c1 + __popc(zero));
        S += (unsigned)(2 * c2 + c1);
        S2 += (unsigned)(4 * c2 + c1);
      }
    }
  } else {
    const int nchunk = (N + 15) >> 4;
#pragma unroll 4
    for (int c = lane; c < nchunk; c += 32) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + c);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
      uint32_t mbits = 0;
      if (mrow) mbits = (mrow[(c * 16) >> 5] >> ((c * 16) & 31)) & 0xFFFFu;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = c * 16 + q * 4 + b;
          const uint32_t u = (w4[q] >> (8 * b)) & 0xFFu;
          if (i < N && !((mbits >> (q * 4 + b)) & 1u)) {
            n += 1;
            S += u;
            S2 += u * u;
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
    float* __restrict__ shift_out, long long lda, int32_t* __restrict__ nobs_out,
    long long* __restrict__ S_out, long long* __restrict__ S2_out, double* __restrict__ mean_out,
    double* __restrict__ gc2_out) {
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
  // pass 2: operand row
  const double m_imp = n ? mean : 0.0;
  const long long steps = lda >> 3;
  if (PREC == TG_PREC_SPLIT_BF16) {
    const double c = row_shift<ENC>(n, mean);
    if (lane == 0 && shift_out) shift_out[j] = (float)c;
    const float cf = (float)c;  // exact: a multiple of 2^-7 in [0, 2] or an integer in [0, 255]
    const __nv_bfloat16 mh = __double2bfloat16(m_imp - c);
    __nv_bfloat16* ah = reinterpret_cast<__nv_bfloat16*>(Ahi) + j * lda;
#pragma unroll 4
    for (long long t = lane; t < steps; t += 32) {
      const int i0 = (int)(t << 3);
      float v[8];
      uint32_t ms = 0;
      __align__(16) __nv_bfloat16 hv[8];
      if (i0 < N) {
        load8<ENC>(row, mrow, i0, N, v, ms);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const bool m = (ms >> s) & 1u;
          // v - c is exact in FP32 and in bf16; samples past N stay 0
          hv[s] = m ? mh : __float2bfloat16_rn(i0 + s < N ? v[s] - cf : 0.0f);
        }
      } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) hv[s] = __float2bfloat16_rn(0.0f);
      }
      *reinterpret_cast<uint4*>(ah + i0) = *reinterpret_cast<const uint4*>(hv);
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

template <int ENC, int PREC>
cudaError_t go(const uint8_t* G, int64_t ldg, int64_t N, int64_t M, const uint32_t* missing,
               int64_t ldm, void* Ahi, float* shift, int64_t lda, int32_t* nobs, int64_t* S,
               int64_t* S2, double* mean, double* gc2, cudaStream_t st) {
  const unsigned grid = (unsigned)((M + kWarps - 1) / kWarps);
  k_decode<ENC, PREC><<<grid, kWarps * 32, 0, st>>>(
      G, ldg, (int)N, M, missing, ldm, Ahi, shift, lda, nobs, reinterpret_cast<long long*>(S),
      reinterpret_cast<long long*>(S2), mean, gc2);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decode(const uint8_t* G, int64_t ldg, int encoding, int64_t N, int64_t M,
                          const uint32_t* missing, int64_t ldm, int precision, void* Ahi,
                          float* shift, int64_t lda, int32_t* nobs, int64_t* S, int64_t* S2,
                          double* mean, double* gc2, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  if (encoding == TG_ENC_2BIT) {
    return precision == TG_PREC_SPLIT_BF16
               ? go<TG_ENC_2BIT, TG_PREC_SPLIT_BF16>(G, ldg, N, M, missing, ldm, Ahi, shift, lda, nobs, S, S2, mean, gc2, st)
               : go<TG_ENC_2BIT, TG_PREC_FP32>(G, ldg, N, M, missing, ldm, Ahi, shift, lda, nobs, S, S2, mean, gc2, st);
  }
  return precision == TG_PREC_SPLIT_BF16
             ? go<TG_ENC_U8_DOSAGE, TG_PREC_SPLIT_BF16>(G, ldg, N, M, missing, ldm, Ahi, shift, lda, nobs, S, S2, mean, gc2, st)
             : go<TG_ENC_U8_DOSAGE, TG_PREC_FP32>(G, ldg, N, M, missing, ldm, Ahi, shift, lda, nobs, S, S2, mean, gc2, st);
}

}  // namespace tg
