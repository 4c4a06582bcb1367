// Device helpers shared by the scan kernels: bounded waits, reductions, epilogue math.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "internal.h"
#include "pvalue.cuh"

namespace tg {

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sum over a whole thread block (any size multiple of 32, <= 1024); every thread gets it.
__device__ __forceinline__ double block_sum(double v, double* red /* >= 33 doubles of smem */) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = (l < nw) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Key of the per-phenotype best marker: larger |r| first, then the smaller marker.
__device__ __forceinline__ unsigned long long best_key(float r, long long marker) {
  if (!(fabsf(r) >= 0.0f)) return 0ull;  // NaN
  return ((unsigned long long)__float_as_uint(fabsf(r)) << 32) |
         (unsigned long long)(0xFFFFFFFFu - (uint32_t)marker);
}

// r from the raw product D of a marker row and a unit-norm phenotype column (NaN kept).
__device__ __forceinline__ float corr_nan(float D, float rinv, float rmul) {
  const float r = D * rinv * rmul;
  if (r != r) return r;
  return fminf(1.0f, fmaxf(-1.0f, r));
}

// Full statistics of one element (FP32, p-value in FP64).
__device__ __forceinline__ void elem_full(const EpiParams& ep, float r, float s_p, float rinv,
                                          float& beta, float& se, float& t, float& mlp) {
  const float omr2 = (1.0f - r) * (1.0f + r);
  const float scale = s_p * rinv / ep.kappa;  // s_p / |g_res| in allele units
  beta = r * scale;
  se = scale * sqrtf(omr2 / ep.df_f);
  t = r * sqrtf(ep.df_f / omr2);
  mlp = (float)mlog10p_r((double)r, ep.df, ep.lnB);
}

// Append one hit (FP64 statistics from the FP32 product D).
__device__ __forceinline__ void emit_hit(const EpiParams& ep, float D, int row, int col) {
  const double rinv = ep.row_inv64[row];
  double r = (double)D * rinv;
  r = fmin(1.0, fmax(-1.0, r));
  const double omr2 = (1.0 - r) * (1.0 + r);
  const double scale = ep.col_s64[col] * rinv / (double)ep.kappa;
  const unsigned long long slot = atomicAdd(ep.n_hits, 1ull);
  if ((long long)slot >= ep.hit_cap) {
    atomicOr(ep.status, ST_CAPACITY);
    return;
  }
  tg_hit h;
  h.marker = (uint32_t)(ep.marker_offset + row);
  h.pheno = (uint32_t)col;
  h.beta = (float)(r * scale);
  h.se = (float)(scale * sqrt(omr2 / ep.df));
  h.t = (float)(r * sqrt(ep.df / omr2));
  h.mlog10p = (float)mlog10p_r(r, ep.df, ep.lnB);
  ep.hits[slot] = h;
}

}  // namespace tg
