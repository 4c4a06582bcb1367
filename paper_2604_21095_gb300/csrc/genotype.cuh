// Conversion of packed genotype codes to the centred split (bf16) operand, shared by the
// decode kernels and the contraction kernels that decode in their producer.
//
// The split operand holds code - c for an observed call (c: the row's shift, a multiple of
// 1/128 for 2-bit calls or an integer for dosage bytes, so the difference is exact in bf16)
// and bf16(mean - c) for a missing call; samples past N are 0.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tg {

// 16 split-form values of 2-bit fields w (sample 16t + k in bits 2k..2k+1): eight bf16x2
// words. lut0 = {field 00, field 01} and lut1 = {field 10, field 11} as bf16 pairs; the
// permute selector for fields (f, g) is 0x1010 + 0x22 f + 0x2200 g (bytes 2f, 2f+1, 2g, 2g+1).
__device__ __forceinline__ void split16_2bit(uint32_t w, uint32_t lut0, uint32_t lut1,
                                             uint32_t (&o)[8]) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint32_t f = (w >> (4 * p)) & 3u, g = (w >> (4 * p + 2)) & 3u;
    o[p] = __byte_perm(lut0, lut1, 0x1010u + 0x22u * f + 0x2200u * g);
  }
}

// 16 split-form values of dosage bytes v: b - c exactly, bf16x2 words; bits of `miss` take
// the missing value mh (a bf16 in the low half of mh2 and in the high half).
__device__ __forceinline__ void split16_u8(uint4 v, float c_plus, uint32_t miss, uint32_t mh2,
                                           uint32_t (&o)[8]) {
  const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint32_t w = w4[p >> 1];
    const uint32_t k = (uint32_t)(p & 1) * 2u;
    const float a = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + k)) - c_plus;
    const float b = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7441u + k)) - c_plus;
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t r = *reinterpret_cast<uint32_t*>(&h);
    const uint32_t m = (miss >> (2 * p)) & 3u;
    if (m) r = __byte_perm(r, mh2, (m & 1u ? 0x0054u : 0x0010u) | (m & 2u ? 0x7600u : 0x3200u));
    o[p] = r;
  }
}

// Zero the values of samples >= N in the 16-sample group starting at i0 (all of them if i0 >= N).
__device__ __forceinline__ void zero_tail16(uint32_t (&o)[8], int i0, int N) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int i = i0 + 2 * p;
    if (i >= N) o[p] = 0u;
    else if (i + 1 >= N) o[p] &= 0xFFFFu;
  }
}

// bf16 bits of x (round to nearest even).
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Exact counts of one 32-bit word of 2-bit fields (16 samples, the first of which is `left`
// samples before N; fields at or past N are ignored): n observed calls, S the sum of their
// allele-1 counts and S2 the sum of squares (field 00 -> 2, 10 -> 1, 11 -> 0, 01 missing).
__device__ __forceinline__ void count16_2bit(uint32_t w, int left, unsigned long long& n,
                                             unsigned long long& S, unsigned long long& S2) {
  if (left <= 0) return;
  const uint32_t valid = (left >= 16) ? 0x55555555u : (0x55555555u & ((1u << (2 * left)) - 1u));
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

}  // namespace tg
