// SIMT kernels: marker projection on Q, marker norms, and the plain FP32 scan.
//
// Projection (a reading of Section 2.2, where the paper only standardises each marker):
// every marker is projected on the covariate basis too, so that the correlation with the
// residualised panel is the exact OLS test. Because every column of the residualised
// panel is orthogonal to Q (intercept included), g_res . y_res = g_imputed . y_res, so the
// contraction can use the imputed codes directly and only the norm needs the projection:
// |g_res|^2 = |g_c|^2 - sum_{k>=1} (q_k . g)^2 (q_0 = the intercept direction drops out).
//
// The FP32 scan is the plain-precision form of Eq. 2: FP32 operands, FP32 FFMA, 128 x 128
// tiles of 8 x 8 per thread, followed by the same fused epilogue as the tensor-core path.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

// ---------------------------------------------------------------- projection
// qg[m][k] = sum_i A[m][i] QB[k][i]; tile 64 markers x 32 columns, 32 samples per step.
__global__ void __launch_bounds__(256) k_project(const float* __restrict__ A, long long lda,
                                                 long long M, int K,
                                                 const float* __restrict__ QB, int nq,
                                                 float* __restrict__ qg) {
  __shared__ __align__(16) float As[32][64 + 4];
  __shared__ __align__(16) float Qs[32][32 + 4];
  const int tid = threadIdx.x;
  const long long m0 = (long long)blockIdx.x * 64;
  const int k0 = blockIdx.y * 32;
  const int tx = tid & 15, ty = tid >> 4;  // 2 columns (k) x 4 markers per thread
  // FP32 partial sums over 256 samples, flushed into FP64 totals
  float acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  double tot[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int i0 = 0; i0 < K; i0 += 32) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {  // A tile: 64 rows x 32 samples as 512 float4
      const int e = tid + u * 256;
      const int r = e >> 3, c4 = (e & 7) * 4;
      const long long gm = m0 + r;
      float4 v = make_float4(0, 0, 0, 0);
      if (gm < M) v = *reinterpret_cast<const float4*>(A + gm * lda + i0 + c4);
      As[c4 + 0][r] = v.x;
      As[c4 + 1][r] = v.y;
      As[c4 + 2][r] = v.z;
      As[c4 + 3][r] = v.w;
    }
    {  // Q tile: 32 columns x 32 samples
      const int r = tid >> 3, c4 = (tid & 7) * 4;
      const float4 v = *reinterpret_cast<const float4*>(QB + (long long)(k0 + r) * K + i0 + c4);
      Qs[c4 + 0][r] = v.x;
      Qs[c4 + 1][r] = v.y;
      Qs[c4 + 2][r] = v.z;
      Qs[c4 + 3][r] = v.w;
    }
    __syncthreads();
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const float4 a = *reinterpret_cast<const float4*>(&As[i][ty * 4]);
      const float2 q = *reinterpret_cast<const float2*>(&Qs[i][tx * 2]);
      acc[0][0] += a.x * q.x; acc[0][1] += a.x * q.y;
      acc[1][0] += a.y * q.x; acc[1][1] += a.y * q.y;
      acc[2][0] += a.z * q.x; acc[2][1] += a.z * q.y;
      acc[3][0] += a.w * q.x; acc[3][1] += a.w * q.y;
    }
    __syncthreads();
    if (((i0 >> 5) & 7) == 7 || i0 + 32 >= K) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          tot[a][b] += (double)acc[a][b];
          acc[a][b] = 0.0f;
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const long long gm = m0 + ty * 4 + a;
    if (gm >= M) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int k = k0 + tx * 2 + b;
      if (k < nq) qg[gm * QCOLS + k] = (float)tot[a][b];
    }
  }
}

// ---------------------------------------------------------------- marker norms
// A marker is re-projected in FP64 (k_marker_refine) when the covariates explain more than
// this share of its variance: |g_res|^2 = |g_c|^2 - sum_k (q_k . g_c)^2 then amplifies the
// rounding of the projections by |g_c|^2 / |g_res|^2 (>= 2 here).
constexpr double kRefineShare = 0.5;

// A marker is tested when it has an observed call, is not constant and its variance inflation
// factor on the covariates, |g_c|^2 / |g_res|^2 = 1 / (1 - R^2 of g on [1, C]), is at most
// kMaxVif: beyond it the covariates explain more than 98% of its variance (the collinearity
// limit PLINK's linear model applies to its predictors by default). Every marker near the
// limit has a ratio far above 1 / (1 - kRefineShare), so its norm is decided in FP64.
constexpr double kMaxVif = 50.0;

__device__ __forceinline__ bool marker_testable(int n_obs, double c2, double r2) {
  return n_obs > 0 && c2 > 0.0 && kMaxVif * r2 >= c2;
}
// complete_n > 0: a marker must also have all complete_n calls observed (the FP4 form, whose
// operand cannot hold a missing call's imputed mean).
__device__ __forceinline__ bool marker_testable(int n_obs, double c2, double r2, int complete_n) {
  return marker_testable(n_obs, c2, r2) && (complete_n <= 0 || n_obs == complete_n);
}

__global__ void k_marker_norm(long long M, const int32_t* __restrict__ nobs,
                              const double* __restrict__ gc2, const float* __restrict__ qg,
                              long long ldq, int nq,
                              double kappa, double* __restrict__ gres2u,
                              double* __restrict__ norm2_allele, float* __restrict__ rinv,
                              double* __restrict__ rinv64, int* __restrict__ refine_list,
                              unsigned* __restrict__ refine_count, int complete_n) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double c2 = gc2[j];
  double s = 0.0;
  for (int k = 0; k < nq; ++k) {
    const double v = (double)qg[j * ldq + k];
    s += v * v;
  }
  const double r2 = c2 - s;
  const bool ok = marker_testable(nobs[j], c2, r2, complete_n);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const double inv = ok ? 1.0 / sqrt(r2) : nan;
  gres2u[j] = ok ? r2 : nan;
  if (norm2_allele) norm2_allele[j] = ok ? r2 * kappa * kappa : nan;
  rinv[j] = (float)inv;
  rinv64[j] = inv;
  if (refine_list && nobs[j] > 0 && c2 > 0.0 && r2 < (1.0 - kRefineShare) * c2)
    refine_list[atomicAdd(refine_count, 1u)] = (int)j;
}

// FP64 re-projection of the listed markers, one block of 256 threads per marker:
// sum_k (q_k . g_c)^2 over the non-intercept columns of Q from the packed genotypes (missing
// calls at the marker's mean, which is also its centre, so they add nothing) and the FP64 mean,
// then the marker's norm outputs again. q_0 . g_c = 0 exactly (q_0 is constant and g_c has zero
// sum), as in the tensor-core projection, which leaves column 0 out.
__global__ void __launch_bounds__(256) k_marker_refine(MarkerRefine rf, const int32_t* __restrict__ nobs,
                                                       const double* __restrict__ gc2, double kappa,
                                                       double* __restrict__ gres2u,
                                                       double* __restrict__ norm2_allele,
                                                       float* __restrict__ rinv,
                                                       double* __restrict__ rinv64,
                                                       int complete_n) {
  __shared__ double red[8];
  const unsigned n = *rf.count;
  for (unsigned li = blockIdx.x; li < n; li += gridDim.x) {
    const long long j = rf.list[li];
    const double mu = rf.mean[j];
    const uint8_t* row = rf.G + j * rf.ldg;
    const uint32_t* mrow = rf.missing ? rf.missing + j * rf.ldm : nullptr;
    double s = 0.0;  // thread 0's copy is the sum
    for (int k = 1; k < rf.q; ++k) {
      const double* qk = rf.Q + (long long)k * rf.N;
      double acc = 0.0;
      for (long long i = threadIdx.x; i < rf.N; i += blockDim.x) {
        double v;
        if (rf.encoding == TG_ENC_2BIT) {
          const unsigned f = (row[i >> 2] >> (2 * (i & 3))) & 3u;  // 00 = 2, 10 = 1, 11 = 0, 01 missing
          v = f == 0u ? 2.0 : f == 2u ? 1.0 : f == 3u ? 0.0 : mu;
        } else {
          const bool miss = mrow && ((mrow[i >> 5] >> (i & 31)) & 1u);
          v = miss ? mu : (double)row[i];
        }
        acc = fma(qk[i], v - mu, acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        s += t * t;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double c2 = gc2[j];
      const double r2 = c2 - s;
      const bool ok = marker_testable(nobs[j], c2, r2, complete_n);
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      const double inv = ok ? 1.0 / sqrt(r2) : nan;
      gres2u[j] = ok ? r2 : nan;
      if (norm2_allele) norm2_allele[j] = ok ? r2 * kappa * kappa : nan;
      rinv[j] = (float)inv;
      rinv64[j] = inv;
    }
  }
}

// ---------------------------------------------------------------- FP32 scan
constexpr int BM = 128, BN = 128, BK = 16;

__global__ void __launch_bounds__(256, 2) k_sgemm_scan(const float* __restrict__ A, long long lda,
                                                    const float* __restrict__ B, long long ldb,
                                                    int K, EpiParams ep) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  __shared__ unsigned long long colbest[BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  // global -> smem mapping: each thread moves 2 float4 of A and 2 of B per K step
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const float* Ag0 = A + (m0 + lr) * lda + lk;
  const float* Ag1 = A + (m0 + lr + 64) * lda + lk;
  const float* Bg0 = B + (long long)(n0 + lr) * ldb + lk;
  const float* Bg1 = B + (long long)(n0 + lr + 64) * ldb + lk;
  if (tid < BN) colbest[tid] = 0ull;

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;

  float4 ra0 = *reinterpret_cast<const float4*>(Ag0);
  float4 ra1 = *reinterpret_cast<const float4*>(Ag1);
  float4 rb0 = *reinterpret_cast<const float4*>(Bg0);
  float4 rb1 = *reinterpret_cast<const float4*>(Bg1);
  int buf = 0;
  auto stash = [&](int bf) {
    As[bf][lk + 0][lr] = ra0.x; As[bf][lk + 1][lr] = ra0.y; As[bf][lk + 2][lr] = ra0.z; As[bf][lk + 3][lr] = ra0.w;
    As[bf][lk + 0][lr + 64] = ra1.x; As[bf][lk + 1][lr + 64] = ra1.y; As[bf][lk + 2][lr + 64] = ra1.z; As[bf][lk + 3][lr + 64] = ra1.w;
    Bs[bf][lk + 0][lr] = rb0.x; Bs[bf][lk + 1][lr] = rb0.y; Bs[bf][lk + 2][lr] = rb0.z; Bs[bf][lk + 3][lr] = rb0.w;
    Bs[bf][lk + 0][lr + 64] = rb1.x; Bs[bf][lk + 1][lr + 64] = rb1.y; Bs[bf][lk + 2][lr + 64] = rb1.z; Bs[bf][lk + 3][lr + 64] = rb1.w;
  };
  stash(0);
  __syncthreads();
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) {
      ra0 = *reinterpret_cast<const float4*>(Ag0 + k0 + BK);
      ra1 = *reinterpret_cast<const float4*>(Ag1 + k0 + BK);
      rb0 = *reinterpret_cast<const float4*>(Bg0 + k0 + BK);
      rb1 = *reinterpret_cast<const float4*>(Bg1 + k0 + BK);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  // epilogue: rows m0 + {ty*4 + a, 64 + ty*4 + a}, columns n0 + {tx*4 + b, 64 + tx*4 + b}
  unsigned long long cb[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) cb[b] = 0ull;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long row = m0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4));
    if (row >= ep.M) continue;
    const float rinv = ep.row_inv[row];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int col = n0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
      if (col >= ep.P) continue;
      const float D = acc[a][b];
      const float r = corr_nan(D, rinv, ep.col_rmul[col]);
      if (ep.do_best) {
        const unsigned long long key = best_key(r, ep.marker_offset + row);
        cb[b] = key > cb[b] ? key : cb[b];
      }
      if (ep.do_hits && r * r >= ep.r2_thr) emit_hit_raw(ep, D, row, col);
      if (ep.do_full) ep.rstore[row * ep.ldo + col] = r;
    }
  }
  if (ep.do_best) {
    // the two ty of a warp share columns: combine, then one shared atomic per column and warp
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, cb[b], 16);
      cb[b] = o > cb[b] ? o : cb[b];
    }
    if ((tid & 16) == 0) {
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int c = b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4);
        if (cb[b]) atomicMax(&colbest[c], cb[b]);
      }
    }
    __syncthreads();
    if (tid < BN && n0 + tid < ep.P && colbest[tid]) best_offer(ep.best + n0 + tid, colbest[tid]);
  }
}

}  // namespace

cudaError_t launch_project(const float* A, int64_t lda, int64_t M, int64_t K, const float* QB,
                           int64_t nq, float* qg, cudaStream_t st) {
  if (M == 0 || nq == 0) return cudaSuccess;
  dim3 grid((unsigned)((M + 63) / 64), (unsigned)((nq + 31) / 32));
  k_project<<<grid, 256, 0, st>>>(A, lda, M, (int)K, QB, (int)nq, qg);
  return cudaGetLastError();
}

cudaError_t launch_marker_norm(int64_t M, const int32_t* nobs, const double* gc2, const float* qg,
                               int64_t ldq, int64_t nq, double kappa, double* gres2_units_out,
                               double* norm2_allele_out, float* rinv, double* rinv64,
                               const MarkerRefine* refine, cudaStream_t st, int64_t complete_n) {
  if (M == 0) return cudaSuccess;
  const bool rf = refine != nullptr && nq > 0;
  if (rf) {
    cudaError_t e = cudaMemsetAsync(refine->count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  k_marker_norm<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(
      M, nobs, gc2, qg, (long long)ldq, (int)nq, kappa, gres2_units_out, norm2_allele_out, rinv, rinv64,
      rf ? refine->list : nullptr, rf ? refine->count : nullptr, (int)complete_n);
  if (!rf) return cudaGetLastError();
  // a fixed grid, so that the launch does not depend on the count (graph capture)
  k_marker_refine<<<304, 256, 0, st>>>(*refine, nobs, gc2, kappa, gres2_units_out,
                                       norm2_allele_out, rinv, rinv64, (int)complete_n);
  return cudaGetLastError();
}

cudaError_t launch_sgemm_scan(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t K,
                              const EpiParams& ep, cudaStream_t st) {
  if (ep.M == 0 || ep.P == 0) return cudaSuccess;
  dim3 grid((unsigned)((ep.P + BN - 1) / BN), (unsigned)((ep.M + BM - 1) / BM));
  k_sgemm_scan<<<grid, 256, 0, st>>>(A, lda, B, ldb, (int)K, ep);
  return cudaGetLastError();
}

}  // namespace tg
