// Panel preparation, run once per phenotype panel (Section 2.1; Section 2.2, Eq. 1).
//
//   1. X = [1, C] (FP64, column-major), with a non-finite check of C.
//   2. Householder QR of X in one thread block: a column whose remaining norm is at most
//      1e-9 of its own norm is dropped (rank detection); Q = H_0 ... H_{q-1} [I_q; 0].
//   3. Per phenotype: Y_res = (I - Q Q^T)(Y - Ybar), s_p = |y_res|, and the unit-norm column
//      y_res / s_p written as FP32 and as a BF16 pair hi = bf16(y), lo = bf16(y - hi).
//   4. Q columns 1..q-1 (the non-intercept directions) in FP32 and as a BF16 pair for the
//      marker projection.
//   5. Per column of the BF16 pairs, sum_i (hi + lo) in FP64: the scan adds c * sum back for a
//      marker row shifted by c (the split operand is centred; see k_decode.cu).
// A panel of phenotypes observed on a subset of the samples is prepared on the gathered rows
// (steps 1-5 with N_S samples) and its sample-indexed arrays are then scattered back to the
// full sample axis with zeros elsewhere (k_gather, k_scatter); k_pheno_masks gives each
// phenotype's finite-value mask, from which such subsets are formed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.h"

namespace tg {
namespace {

constexpr double kRankTol = 1e-9;
constexpr double kPhenoTol = 1e-12;

__global__ void k_build_design(double* __restrict__ X, const double* __restrict__ C, long long ldc,
                               long long N, int n_cov, uint32_t* flags) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  X[i] = 1.0;
  bool bad = false;
  for (int k = 0; k < n_cov; ++k) {
    const double v = C[k * ldc + i];
    bad |= !isfinite(v);
    X[(long long)(k + 1) * N + i] = v;
  }
  if (bad) atomicOr(flags, 1u);
}

// One block of 1024 threads. X [k][N] is reduced in place; V keeps the reflectors.
__global__ void __launch_bounds__(1024) k_householder(double* __restrict__ X, long long N, int k,
                                                       double* __restrict__ V,
                                                       double* __restrict__ Q, int* rank_out,
                                                       int* kept_out) {
  __shared__ double red[33];
  __shared__ double own[QMAX];
  __shared__ int vrow[QMAX];
  __shared__ double vbeta[QMAX];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < k; ++j) {
    double s = 0.0;
    for (long long i = tid; i < N; i += nt) s += X[j * N + i] * X[j * N + i];
    s = block_sum(s, red);
    if (tid == 0) own[j] = sqrt(s);
  }
  __syncthreads();
  int row = 0, q = 0;
  for (int j = 0; j < k && row < N; ++j) {
    double* x = X + (long long)j * N;
    double s = 0.0;
    for (long long i = row + tid; i < N; i += nt) s += x[i] * x[i];
    s = block_sum(s, red);
    const double nrm = sqrt(s);
    if (own[j] == 0.0 || nrm <= kRankTol * own[j]) {
      if (tid == 0) kept_out[j] = 0;
      continue;
    }
    const double x0 = x[row];
    const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
    // v = x + sg |x| e_row (rows >= row); |v|^2 = 2 |x|^2 + 2 |x0| |x|
    double* v = V + (long long)q * N;
    for (long long i = row + tid; i < N; i += nt) v[i] = (i == row) ? x0 + sg * nrm : x[i];
    const double beta = 2.0 / (2.0 * s + 2.0 * fabs(x0) * nrm);
    __syncthreads();
    for (int c = j + 1; c < k; ++c) {
      double* xc = X + (long long)c * N;
      double d = 0.0;
      for (long long i = row + tid; i < N; i += nt) d += v[i] * xc[i];
      d = block_sum(d, red) * beta;
      for (long long i = row + tid; i < N; i += nt) xc[i] -= d * v[i];
      __syncthreads();
    }
    if (tid == 0) {
      kept_out[j] = 1;
      vrow[q] = row;
      vbeta[q] = beta;
    }
    __syncthreads();
    ++row;
    ++q;
  }
  // Q[:, c] = H_0 ... H_{q-1} e_c, applying the reflectors in reverse order.
  for (int c = 0; c < q; ++c)
    for (long long i = tid; i < N; i += nt) Q[(long long)c * N + i] = (i == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int r = q - 1; r >= 0; --r) {
    const double* v = V + (long long)r * N;
    const long long r0 = vrow[r];
    const double beta = vbeta[r];
    for (int c = r; c < q; ++c) {
      double* qc = Q + (long long)c * N;
      double d = 0.0;
      for (long long i = r0 + tid; i < N; i += nt) d += v[i] * qc[i];
      d = block_sum(d, red) * beta;
      for (long long i = r0 + tid; i < N; i += nt) qc[i] -= d * v[i];
      __syncthreads();
    }
  }
  if (tid == 0) *rank_out = q;
}

// One block per phenotype column.
__global__ void __launch_bounds__(256) k_residualise(
    const float* __restrict__ Y, long long ldy, const double* __restrict__ Q, long long N, int q,
    long long Npad, double* __restrict__ Yres, double* __restrict__ s_out, float* __restrict__ col_s,
    float* __restrict__ col_rmul, __nv_bfloat16* __restrict__ Bhi, __nv_bfloat16* __restrict__ Blo,
    float* __restrict__ B32, float* __restrict__ col_cs, uint32_t* flags) {
  __shared__ double red[33];
  __shared__ double coef[QMAX];
  const long long p = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const float* y = Y + p * ldy;
  double* yr = Yres + p * N;
  // mean and finiteness
  double sum = 0.0;
  bool bad = false;
  for (long long i = tid; i < N; i += nt) {
    const double v = (double)y[i];
    bad |= !isfinite(v);
    sum += v;
  }
  if (bad) atomicOr(flags, 2u);
  const double ybar = block_sum(sum, red) / (double)N;
  // coefficients Q^T (y - ybar), eight at a time
  for (int k0 = 0; k0 < q; k0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (long long i = tid; i < N; i += nt) {
      const double yc = (double)y[i] - ybar;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < q) acc[u] += Q[(long long)(k0 + u) * N + i] * yc;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (k0 + u < q) {
        const double c = block_sum(acc[u], red);
        if (tid == 0) coef[k0 + u] = c;
      }
    }
  }
  __syncthreads();
  // residual, its norm and the centred norm
  double rs = 0.0, cs = 0.0;
  for (long long i = tid; i < N; i += nt) {
    const double yc = (double)y[i] - ybar;
    double r = yc;
    for (int k = 0; k < q; ++k) r -= Q[(long long)k * N + i] * coef[k];
    yr[i] = r;
    rs += r * r;
    cs += yc * yc;
  }
  rs = block_sum(rs, red);
  cs = block_sum(cs, red);
  const double s = sqrt(rs);
  const bool ok = s > kPhenoTol * sqrt(cs);
  if (tid == 0) {
    s_out[p] = s;
    col_s[p] = ok ? (float)s : __int_as_float(0x7fc00000);
    col_rmul[p] = ok ? 1.0f : __int_as_float(0x7fc00000);
  }
  const double inv = ok ? 1.0 / s : 0.0;
  __nv_bfloat16* bh = Bhi + p * Npad;
  __nv_bfloat16* bl = Blo + p * Npad;
  float* bf = B32 + p * Npad;
  double bsum = 0.0;
  for (long long i = tid; i < Npad; i += nt) {
    const double u = (i < N) ? yr[i] * inv : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(u);
    const __nv_bfloat16 l = __double2bfloat16(u - (double)__bfloat162float(h));
    bh[i] = h;
    bl[i] = l;
    bf[i] = (float)u;
    bsum += (double)__bfloat162float(h) + (double)__bfloat162float(l);
  }
  bsum = block_sum(bsum, red);
  if (tid == 0) col_cs[p] = (float)bsum;
}

// Row sums of the bf16 pair of the projection columns.
__global__ void __launch_bounds__(256) k_qcolsum(const __nv_bfloat16* __restrict__ QBhi,
                                                 const __nv_bfloat16* __restrict__ QBlo,
                                                 long long Npad, float* __restrict__ qcs) {
  __shared__ double red[33];
  const long long r = blockIdx.x;
  double cs = 0.0;
  for (long long i = threadIdx.x; i < Npad; i += blockDim.x)
    cs += (double)__bfloat162float(QBhi[r * Npad + i]) + (double)__bfloat162float(QBlo[r * Npad + i]);
  cs = block_sum(cs, red);
  if (threadIdx.x == 0) qcs[r] = (float)cs;
}

__global__ void k_qcols(const double* __restrict__ Q, long long N, int q, long long Npad,
                        float* __restrict__ QB, __nv_bfloat16* __restrict__ QBhi,
                        __nv_bfloat16* __restrict__ QBlo) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;  // QB row r = Q column r + 1
  if (i >= Npad) return;
  const double v = (r + 1 < q && i < N) ? Q[(long long)(r + 1) * N + i] : 0.0;
  const long long o = (long long)r * Npad + i;
  QB[o] = (float)v;
  const __nv_bfloat16 h = __double2bfloat16(v);
  QBhi[o] = h;
  QBlo[o] = __double2bfloat16(v - (double)__bfloat162float(h));
}

// The joint operand of a small panel in f16, for the joint pass that decodes dosage rows in
// shared memory (k_fused.cu): rows [0, nq) = Q columns 1..nq, rows [nq, nq + P) = the unit-norm
// residualised phenotypes (0 for an untestable one), the rest 0; each value v (|v| <= 1) scaled
// by 2^14 and split into hi = f16(2^14 v), lo = f16(2^14 v - hi), about 22 significant bits
// (|2^14 v| <= 16,384, inside f16's range, and lo stays a normal number down to |v| ~ 2^-25).
// cs[r] = sum_i (hi + lo) in FP64, rounded to FP32, the scaled column sum of the shift add-back.
__global__ void __launch_bounds__(256) k_joint_f16(const double* __restrict__ Q, long long N, int nq,
                                                   const double* __restrict__ Yres,
                                                   const double* __restrict__ s,
                                                   const float* __restrict__ rmul, int P,
                                                   long long Npad, __half* __restrict__ hi,
                                                   __half* __restrict__ lo, float* __restrict__ cs) {
  __shared__ double red[33];
  const int r = blockIdx.x;
  const double* src = nullptr;
  double mul = 0.0;
  if (r < nq) {
    src = Q + (long long)(r + 1) * N;
    mul = kJointF16Scale;
  } else if (r < nq + P) {
    const int p = r - nq;
    if (rmul[p] == rmul[p]) {  // a testable phenotype: y_res / s, as the bf16 panel
      src = Yres + (long long)p * N;
      mul = (1.0 / s[p]) * kJointF16Scale;
    }
  }
  double sum = 0.0;
  for (long long i = threadIdx.x; i < Npad; i += blockDim.x) {
    const double u = (src && i < N) ? src[i] * mul : 0.0;
    const __half h = __double2half(u);
    const __half l = __double2half(u - (double)__half2float(h));
    hi[(long long)r * Npad + i] = h;
    lo[(long long)r * Npad + i] = l;
    sum += (double)__half2float(h) + (double)__half2float(l);
  }
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) cs[r] = (float)sum;
}

// dst[r][i] = src[r * lds + idx[i]] for r < R, i < ns (rows of a compact copy).
template <class T>
__global__ void k_gather(const T* __restrict__ src, long long lds, T* __restrict__ dst, long long ldd,
                         const int* __restrict__ idx, int ns, int R) {
  const long long total = (long long)R * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ns;
    const int i = (int)(e - r * ns);
    dst[r * ldd + i] = src[r * lds + idx[i]];
  }
}

// dst[r * ldd + idx[i]] = src[r][i] (dst zeroed beforehand).
template <class T>
__global__ void k_scatter(const T* __restrict__ src, long long lds, T* __restrict__ dst, long long ldd,
                          const int* __restrict__ idx, int ns, int R) {
  const long long total = (long long)R * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ns;
    const int i = (int)(e - r * ns);
    dst[r * ldd + idx[i]] = src[r * lds + i];
  }
}

// masks[p][w] bit b = Y[p][32 w + b] is finite (bits past N are 0).
__global__ void k_pheno_masks(const float* __restrict__ Y, long long ldy, long long N, long long P,
                              uint32_t* __restrict__ masks, long long ldm) {
  const long long nw = (N + 31) / 32;
  const long long total = P * nw;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / nw, w = e - p * nw;
    uint32_t m = 0;
    for (int b = 0; b < 32; ++b) {
      const long long i = 32 * w + b;
      if (i < N && isfinite(Y[p * ldy + i])) m |= 1u << b;
    }
    masks[p * ldm + w] = m;
  }
}

template <class T>
unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_gather_f32(const float* src, int64_t lds, float* dst, int64_t ldd, const int* idx,
                              int64_t ns, int64_t R, cudaStream_t st) {
  if (ns == 0 || R == 0) return cudaSuccess;
  k_gather<float><<<grid_for<float>(R * ns), 256, 0, st>>>(src, lds, dst, ldd, idx, (int)ns, (int)R);
  return cudaGetLastError();
}
cudaError_t launch_gather_f64(const double* src, int64_t lds, double* dst, int64_t ldd,
                              const int* idx, int64_t ns, int64_t R, cudaStream_t st) {
  if (ns == 0 || R == 0) return cudaSuccess;
  k_gather<double><<<grid_for<double>(R * ns), 256, 0, st>>>(src, lds, dst, ldd, idx, (int)ns, (int)R);
  return cudaGetLastError();
}
cudaError_t launch_scatter(const void* src, int64_t lds, void* dst, int64_t ldd, const int* idx,
                           int64_t ns, int64_t R, int elem_bytes, cudaStream_t st) {
  if (ns == 0 || R == 0) return cudaSuccess;
  const unsigned g = grid_for<char>(R * ns);
  if (elem_bytes == 8)
    k_scatter<double><<<g, 256, 0, st>>>(static_cast<const double*>(src), lds, static_cast<double*>(dst), ldd, idx, (int)ns, (int)R);
  else if (elem_bytes == 4)
    k_scatter<float><<<g, 256, 0, st>>>(static_cast<const float*>(src), lds, static_cast<float*>(dst), ldd, idx, (int)ns, (int)R);
  else if (elem_bytes == 2)
    k_scatter<unsigned short><<<g, 256, 0, st>>>(static_cast<const unsigned short*>(src), lds, static_cast<unsigned short*>(dst), ldd, idx, (int)ns, (int)R);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t launch_pheno_masks(const float* Y, int64_t ldy, int64_t N, int64_t P, uint32_t* masks,
                               int64_t ldm, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_pheno_masks<<<grid_for<char>(P * ((N + 31) / 32)), 256, 0, st>>>(Y, ldy, N, P, masks, ldm);
  return cudaGetLastError();
}

cudaError_t launch_build_design(double* X, const double* C, int64_t ldc, int64_t N, int64_t n_cov,
                                uint32_t* flags, cudaStream_t st) {
  const int tb = 256;
  k_build_design<<<(unsigned)((N + tb - 1) / tb), tb, 0, st>>>(X, C, ldc, N, (int)n_cov, flags);
  return cudaGetLastError();
}

cudaError_t launch_householder(double* X, int64_t N, int64_t k, double* Q, int* rank_out,
                               int* kept_out, cudaStream_t st) {
  // The reflectors are stored after the k columns of X (the caller allocates 2k columns).
  k_householder<<<1, 1024, 0, st>>>(X, N, (int)k, X + k * N, Q, rank_out, kept_out);
  return cudaGetLastError();
}

cudaError_t launch_residualise(const float* Y, int64_t ldy, const double* Q, int64_t N, int64_t P,
                               int64_t q, int64_t Npad, double* Yres, double* s, float* col_s,
                               float* col_rmul, __nv_bfloat16* Bhi, __nv_bfloat16* Blo, float* B32,
                               float* col_cs, uint32_t* flags, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_residualise<<<(unsigned)P, 256, 0, st>>>(Y, ldy, Q, N, (int)q, Npad, Yres, s, col_s, col_rmul,
                                             Bhi, Blo, B32, col_cs, flags);
  return cudaGetLastError();
}

cudaError_t launch_joint_f16(const double* Q, int64_t N, int64_t nq, const double* Yres,
                             const double* s, const float* rmul, int64_t P, int64_t rows,
                             int64_t Npad, __half* hi, __half* lo, float* cs, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_joint_f16<<<(unsigned)rows, 256, 0, st>>>(Q, N, (int)nq, Yres, s, rmul, (int)P, Npad, hi, lo, cs);
  return cudaGetLastError();
}

cudaError_t launch_qcols(const double* Q, int64_t N, int64_t q, int64_t Npad, float* QB,
                         __nv_bfloat16* QBhi, __nv_bfloat16* QBlo, float* qcs, cudaStream_t st) {
  dim3 grid((unsigned)((Npad + 255) / 256), QCOLS);
  k_qcols<<<grid, 256, 0, st>>>(Q, N, (int)q, Npad, QB, QBhi, QBlo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_qcolsum<<<QCOLS, 256, 0, st>>>(QBhi, QBlo, Npad, qcs);
  return cudaGetLastError();
}

}  // namespace tg
