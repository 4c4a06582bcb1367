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

// Offer a key to a per-phenotype best: a global max reduction that returns nothing, so the
// thread does not wait for the round trip (atomicMax would).
__device__ __forceinline__ void best_offer(unsigned long long* best, unsigned long long key) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(best), "l"(key) : "memory");
}

// r from the raw product D of a marker row and a unit-norm phenotype column (NaN kept).
__device__ __forceinline__ float corr_nan(float D, float rinv, float rmul) {
  const float r = D * rinv * rmul;
  if (r != r) return r;
  return fminf(1.0f, fmaxf(-1.0f, r));
}

// Append a raw hit record: marker, phenotype and the product D (in the beta slot). The
// statistics kernel that runs after the contraction turns it into beta, se, t, -log10 p.
__device__ __forceinline__ void emit_hit_raw(const EpiParams& ep, float D, long long row, int col) {
  const unsigned long long slot = atomicAdd(ep.n_hits, 1ull);
  if (slot >= (unsigned long long)ep.hit_cap) {  // unsigned: any count past capacity, never a write
    atomicOr(ep.status, ST_CAPACITY);
    return;
  }
  tg_hit h;
  h.marker = (uint32_t)(ep.marker_offset + row);
  h.pheno = (uint32_t)col;
  h.beta = D;
  h.se = 0.0f;
  h.t = 0.0f;
  h.mlog10p = 0.0f;
  ep.hits[slot] = h;
}

}  // namespace tg
