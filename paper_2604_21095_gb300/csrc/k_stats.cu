// Statistics of Eq. 3 and the P value, after the contraction (Section 2.2).
//
// The contraction epilogues only keep what needs the accumulator: r for every element in FULL
// mode (stored in one of the caller's output arrays) and raw hit records (marker, phenotype,
// product D). These kernels turn them into
//   t = r sqrt(df / ((1 - r)(1 + r))),  beta = r s_p / (kappa |a_res|),
//   se = s_p / (kappa |a_res|) sqrt((1 - r)(1 + r) / df),  -log10 p with p = I_{1-r^2}(df/2, 1/2).
// Every hit, and every FULL element whose 1 - r^2 is below kExactOmr2, is recomputed in FP64:
// the product g_j . y_res,p from the packed genotype row (missing calls at the FP64 mean) and
// the panel's FP64 residualised phenotype, r from it and the FP64 marker norm, and -log10 p
// in FP64 (the continued fraction, or Hill's deviate where that is within 0.05 of the
// tolerance and the fraction converges slowly; pvalue.cuh). Near |r| = 1 the p-value's slope in r, df / (1 - r^2),
// turns the FP32 product's rounding into errors above the tolerance (see kExactOmr2). The
// other FULL elements take their p-values in FP32 log space (see pvalue.cuh).
#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

// sum over this thread's groups of 8 samples (8t, 8(t + nt), ...) of (g_i - mean) y_res,p,i in
// FP64, for the marker in block row `row` (the centring adds nothing, since y_res,p sums to zero,
// but keeps the terms small). The eight loads of a group are issued before any is used, so that
// a few hundred threads keep enough loads in flight to stream the 8 N bytes of y_res,p.
__device__ __forceinline__ double exact_partial(const ExactArgs& x, long long row, int col, int t,
                                                int nt) {
  const uint8_t* g = x.G + row * x.ldg;
  const uint32_t* mrow = x.missing ? x.missing + row * x.ldm : nullptr;
  const double mu = x.mean[row];
  const double* y = x.Yres + (long long)col * x.ldy;
  // 2-bit fields 00 (2 copies), 10 (1), 11 (0) minus the mean; 01 (missing) is the mean itself
  const double c00 = 2.0 - mu, c10 = 1.0 - mu, c11 = -mu;
  double acc0 = 0.0, acc1 = 0.0;
  for (int i0 = 8 * t; i0 < x.N; i0 += 8 * nt) {
    const bool whole = i0 + 8 <= x.N;
    double yv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) yv[u] = (whole || i0 + u < x.N) ? y[i0 + u] : 0.0;
    double v[8];
    if (x.encoding == TG_ENC_2BIT) {  // samples i0..i0+7 in bytes i0/4 and i0/4 + 1
      const unsigned w = (unsigned)g[i0 >> 2] | ((i0 + 4 < x.N ? (unsigned)g[(i0 >> 2) + 1] : 0u) << 8);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const unsigned f = (w >> (2 * u)) & 3u;
        v[u] = f == 0u ? c00 : f == 2u ? c10 : f == 3u ? c11 : 0.0;
      }
    } else {
      uint2 b = make_uint2(0u, 0u);
      if (whole) {
        b = *reinterpret_cast<const uint2*>(g + i0);  // row starts 16-byte aligned, i0 % 8 == 0
      } else {
        for (int u = 0; i0 + u < x.N; ++u) (u < 4 ? b.x : b.y) |= (unsigned)g[i0 + u] << (8 * (u & 3));
      }
      const unsigned mb = mrow ? (mrow[i0 >> 5] >> (i0 & 31)) & 0xFFu : 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const unsigned byte = ((u < 4 ? b.x : b.y) >> (8 * (u & 3))) & 0xFFu;
        v[u] = ((mb >> u) & 1u) ? 0.0 : (double)byte - mu;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      acc0 = fma(v[u], yv[u], acc0);
      acc1 = fma(v[u + 1], yv[u + 1], acc1);
    }
  }
  return acc0 + acc1;
}

// The FP64 statistics of one element from its FP64 product D = g . y_res,p (decode units).
struct Stats64 {
  float beta, se, t, mlp;
};
__device__ __forceinline__ Stats64 stats_exact(const EpiParams& ep, long long row, int col, double D) {
  const double s = ep.col_s64[col];
  const double rinv = ep.row_inv64[row];
  double r = D / s * rinv;
  r = fmin(1.0, fmax(-1.0, r));
  const double omr2 = (1.0 - r) * (1.0 + r);
  const double scale = s * rinv / ep.kappa64;
  Stats64 o;
  o.beta = (float)(r * scale);
  o.se = (float)(scale * sqrt(omr2 / ep.df));
  o.t = (float)(r * sqrt(ep.df / omr2));
  o.mlp = (float)mlog10p_r_dev(r, ep.df, ep.lnB);
  return o;
}

// FULL statistics. Each warp walks 32 consecutive elements at a time (all lanes stay in the
// loop), so that the rare elements near |r| = 1 can be recomputed by the whole warp.
__global__ void __launch_bounds__(256, 1) k_full_stats(EpiParams ep) {
  const long long total = (long long)ep.M * ep.P;
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < total;
       base += wstride) {
    const long long e = base + lane;
    long long row = 0, o = 0;
    int col = 0;
    bool exact = false;
    if (e < total) {
      row = e / ep.P;
      col = (int)(e - row * ep.P);
      o = row * ep.ldo + col;
      const float r = ep.rstore[o];
      const float omr2 = (1.0f - r) * (1.0f + r);
      exact = ep.exact.G != nullptr && omr2 < kExactOmr2;  // false for NaN
      if (!exact) {
        const float rinv = ep.row_inv[row];
        const float scale = ep.col_s[col] * rinv / ep.kappa;
        if (ep.beta) ep.beta[o] = r * scale;
        if (ep.se) ep.se[o] = scale * sqrtf(omr2 / ep.df_f);
        if (ep.t) ep.t[o] = r * sqrtf(ep.df_f / omr2);
        if (ep.mlp) ep.mlp[o] = mlog10p_r_f(r, ep.df_f, (float)ep.lnB);
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, exact);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const long long xrow = __shfl_sync(0xffffffffu, row, src);
      const int xcol = __shfl_sync(0xffffffffu, col, src);
      double D = exact_partial(ep.exact, xrow, xcol, lane, 32);
      for (int k = 16; k > 0; k >>= 1) D += __shfl_xor_sync(0xffffffffu, D, k);
      if (lane == src) {
        const Stats64 v = stats_exact(ep, row, col, D);
        if (ep.beta) ep.beta[o] = v.beta;
        if (ep.se) ep.se[o] = v.se;
        if (ep.t) ep.t[o] = v.t;
        if (ep.mlp) ep.mlp[o] = v.mlp;
      }
    }
  }
}

// Hit records: one block per hit recomputes its product in FP64 and writes the FP64 statistics.
constexpr int kHitThreads = 512;
__global__ void __launch_bounds__(kHitThreads) k_hit_stats(EpiParams ep,
                                                   const unsigned long long* __restrict__ start) {
  __shared__ double red[33];
  const unsigned long long s0 = *start;
  unsigned long long s1 = *ep.n_hits;
  if (s1 > (unsigned long long)ep.hit_cap) s1 = (unsigned long long)ep.hit_cap;
  for (unsigned long long i = s0 + blockIdx.x; i < s1; i += gridDim.x) {
    tg_hit h = ep.hits[i];
    const long long row = (long long)h.marker - ep.marker_offset;
    const double D = block_sum(exact_partial(ep.exact, row, (int)h.pheno, threadIdx.x, blockDim.x), red);
    if (threadIdx.x == 0) {
      const Stats64 v = stats_exact(ep, row, (int)h.pheno, D);
      h.beta = v.beta;
      h.se = v.se;
      h.t = v.t;
      h.mlog10p = v.mlp;
      ep.hits[i] = h;
    }
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
  if (grid > 152 * 32) grid = 152 * 32;  // a grid-stride loop: 32 blocks per SM at most
  k_full_stats<<<(unsigned)grid, 256, 0, st>>>(ep);
  return cudaGetLastError();
}

cudaError_t launch_hit_stats(const EpiParams& ep, const unsigned long long* start, cudaStream_t st) {
  if (ep.exact.G == nullptr) return cudaErrorInvalidValue;  // hits are always recomputed in FP64
  k_hit_stats<<<152 * 2, kHitThreads, 0, st>>>(ep, start);
  return cudaGetLastError();
}

}  // namespace tg
