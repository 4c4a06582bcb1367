// Statistics of Eq. 3 and the P value, after the contraction (Section 2.2).
//
// The contraction epilogues only keep what needs the accumulator: r for every element in FULL
// mode (stored in one of the caller's output arrays) and raw hit records (marker, phenotype,
// product D). These kernels turn them into
//   t = r sqrt(df / ((1 - r)(1 + r))),  beta = r s_p / (kappa |a_res|),
//   se = s_p / (kappa |a_res|) sqrt((1 - r)(1 + r) / df),  -log10 p with p = I_{1-r^2}(df/2, 1/2).
// Hit records are recomputed from D with FP64 r, beta and se; the p-values (of hits and of
// FULL elements) are evaluated in FP32 log space (see pvalue.cuh).
#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

__global__ void __launch_bounds__(256) k_full_stats(EpiParams ep) {
  const long long total = (long long)ep.M * ep.P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ep.P;
    const int col = (int)(e - row * ep.P);
    const long long o = row * ep.ldo + col;
    const float r = ep.rstore[o];
    const float rinv = ep.row_inv[row];
    const float omr2 = (1.0f - r) * (1.0f + r);
    const float scale = ep.col_s[col] * rinv / ep.kappa;
    if (ep.beta) ep.beta[o] = r * scale;
    if (ep.se) ep.se[o] = scale * sqrtf(omr2 / ep.df_f);
    if (ep.t) ep.t[o] = r * sqrtf(ep.df_f / omr2);
    if (ep.mlp) ep.mlp[o] = mlog10p_r_f(r, ep.df_f, (float)ep.lnB);
  }
}

__global__ void __launch_bounds__(128) k_hit_stats(EpiParams ep,
                                                   const unsigned long long* __restrict__ start) {
  const unsigned long long s0 = *start;
  unsigned long long s1 = *ep.n_hits;
  if (s1 > (unsigned long long)ep.hit_cap) s1 = (unsigned long long)ep.hit_cap;
  for (unsigned long long i = s0 + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       i < s1; i += (unsigned long long)gridDim.x * blockDim.x) {
    tg_hit h = ep.hits[i];
    const long long row = (long long)h.marker - ep.marker_offset;
    const double rinv = ep.row_inv64[row];
    double r = (double)h.beta * rinv;
    r = fmin(1.0, fmax(-1.0, r));
    const double omr2 = (1.0 - r) * (1.0 + r);
    const double scale = ep.col_s64[h.pheno] * rinv / ep.kappa64;
    h.beta = (float)(r * scale);
    h.se = (float)(scale * sqrt(omr2 / ep.df));
    h.t = (float)(r * sqrt(ep.df / omr2));
    h.mlog10p = mlog10p_r_f((float)r, ep.df_f, (float)ep.lnB);
    ep.hits[i] = h;
  }
}

// Deterministic pseudo-random bytes (SplitMix64 of the index); used for timing trial blocks.
__global__ void k_fill_random(uint8_t* __restrict__ p, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    p[i] = (uint8_t)((z ^ (z >> 31)) >> 24);
  }
}

}  // namespace

cudaError_t launch_fill_random(uint8_t* p, size_t n, unsigned long long seed, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_fill_random<<<152 * 8, 256, 0, st>>>(p, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_full_stats(const EpiParams& ep, cudaStream_t st) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  const long long total = (long long)ep.M * ep.P;
  long long grid = (total + 255) / 256;
  if (grid > 148 * 32) grid = 148 * 32;
  k_full_stats<<<(unsigned)grid, 256, 0, st>>>(ep);
  return cudaGetLastError();
}

cudaError_t launch_hit_stats(const EpiParams& ep, const unsigned long long* start, cudaStream_t st) {
  k_hit_stats<<<64, 128, 0, st>>>(ep, start);
  return cudaGetLastError();
}

}  // namespace tg
