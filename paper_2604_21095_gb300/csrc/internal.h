// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tg.h"

namespace tg {

// Latched device status bits (ctx->status).
enum : uint32_t { ST_CAPACITY = 1u, ST_TIMEOUT = 2u };

constexpr int KPAD = 64;     // sample dimension (GEMM K) padding of every operand row
constexpr int kAccumChunkKB = 32;  // tensor-core accumulation chunk: 32 K blocks of 32 samples
constexpr int PPAD = 256;    // phenotype rows padding of the panel operands (tensor-core N tile)
constexpr int QMAX = 64;     // intercept + at most 63 covariates
constexpr int kMaxHostBufs = 4;  // block buffers of the host-streamed scan, at most
// blocks of the host-streamed scan in flight at once (their scan-done events), at most
constexpr int kRingEvents = 8 * kMaxHostBufs + 8;
// blocks of a host-streamed scan (the second to the ninth) whose copies and scans are timed for
// the next call's block growth
constexpr int kRateBlocks = 8;
constexpr int QCOLS = 64;    // projection columns (Q columns 1..q-1), zero padded
constexpr int JCOLS = 256;   // widest joint operand: projection columns + panel in one tile
constexpr int MT = 128;      // marker rows per tensor-core tile
constexpr int kFp4Pieces = 6;  // E2M1 pieces of the panel in the FP4 form (k_fp4.cu)
// Scale of the f16 joint operand (k_joint_f16): values of at most 1 in magnitude become at most
// 2^14, inside f16's range, with the low piece a normal number for |v| >= ~2^-25.
constexpr double kJointF16Scale = 16384.0;

enum Stage { STAGE_DECODE = 0, STAGE_PROJECT = 1, STAGE_NORM = 2, STAGE_GEMM = 3, STAGE_H2D = 4,
             STAGE_STATS = 5 };

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// What the FP64 recomputation of a product g_j . y_res,p needs (hits, and FULL elements near
// |r| = 1): the packed genotype block, its FP64 observed means (decode units; a missing call is
// imputed with it) and the panel's FP64 residualised phenotypes [P][ldy]. G = NULL: off.
struct ExactArgs {
  const uint8_t* G;
  long long ldg;
  int encoding;
  int N;
  const uint32_t* missing;  // dosage mask [M][ldm] or NULL
  long long ldm;
  const double* mean;       // [M]
  const double* Yres;       // [P][ldy], zero outside a subset panel's samples
  long long ldy;
};

// FULL elements whose FP32 1 - r^2 is below this are recomputed in FP64 (hits always are):
// r from the FP32 product carries an absolute error of up to ~5e-7, and d(-log10 p)/dr =
// df |r| / ((1 - r^2) ln 10) makes that exceed the 1e-5 relative tolerance on -log10 p once
// (1 - r^2) ln(1 / (1 - r^2)) < ~0.1, i.e. 1 - r^2 < ~0.03, at every df.
constexpr float kExactOmr2 = 0.05f;

// Per-element statistics inputs shared by both contraction kernels' epilogues.
struct EpiParams {
  int M, P;                    // block rows (markers) and panel phenotypes
  long long marker_offset;
  double df;                   // N - q - 1
  float df_f;
  double lnB;                  // ln Beta(df/2, 1/2)
  float kappa;                 // allele units per decode unit (1 or 2/255), FP32 kernels
  double kappa64;              // the same in FP64 (hit statistics)
  float r2_thr;                // hit threshold on r^2 (> 1 disables)
  int do_full, do_hits, do_best;
  const float* row_inv;        // [M] 1/|a_res| (decode units), NaN = untestable
  const double* row_inv64;     // [M]
  const float* col_s;          // [P] s_p, NaN = untestable phenotype
  const double* col_s64;       // [P]
  const float* col_rmul;       // [P] 1 or NaN
  const float* row_shift;      // [M] c the operand row was shifted by (NULL = none)
  const float* col_cs;         // [P] sum_i of the B operand column (the shift's add-back)
  float *beta, *se, *t, *mlp;  // FULL outputs, [M][ldo]
  float* rstore;               // FULL mode: where the contraction leaves r (one of the above)
  long long ldo;
  tg_hit* hits;
  long long hit_cap;
  unsigned long long* n_hits;
  unsigned long long* best;
  uint32_t* status;
  unsigned long long* wave_ctr;  // CTA-pair lockstep counter (zeroed per launch), NULL = off
  float* raw_out;              // projection mode: D of the first raw_cols columns, [M][raw_ld]
  int raw_cols, raw_ld;
  // split-K (one-CTA kernel): K split in `ksplit` chunk-aligned ranges (0 or 1 = none); the
  // partial sums of splits 1.. go through sk_ws ([tiles][ksplit-1][128][256] floats) and
  // sk_cnt ([tiles], zeroed per launch) to the tile's split 0, which adds them in split order
  int ksplit;
  float* sk_ws;
  unsigned* sk_cnt;
  ExactArgs exact;             // FP64 recomputation of hits and of FULL elements near |r| = 1
};

// Packed genotypes for a contraction kernel that decodes its A operand in the producer
// (2-bit calls, or dosage bytes without a missing mask; split form only). The kernel loads the
// packed rows through `tmG` (uint8, {ldg, M}, boxes of 32 or 16 bytes x 128 rows).
constexpr int kOnePassMaxN = 66051;  // 255^2 * N < 2^32
struct DecodeArgs {
  CUtensorMap tmG;
  int N;                  // samples; K columns >= N are zero
  int M;                  // rows of the block; rows >= M are zero
  const float* shift;     // [M] row shift c
  const uint32_t* mh;     // [M] bf16 bits of (mean - c), the missing-call value
  // Dosage rows without a mask in the joint pass on 256-row tiles: when shift_out is set, the
  // pass takes each row's shift from the row's first 64 samples instead of reading `shift`, sums
  // the row's bytes and their squares as it expands them, and writes the row's statistics (the
  // counting pass's outputs: n_obs = N, mean, |g_c|^2 and the shift), so no counting pass runs.
  float* shift_out;  // (N <= kOnePassMaxN: the sum of squared bytes fits 32 bits)
  int32_t* nobs_out;
  double* mean_out;
  double* gc2_out;
  // The projection pass of a larger panel (the 64 projection columns alone): when a_out is set,
  // the pass also stores each expanded row as the block's bf16 operand (row-major, lda_out
  // elements per row, every column of rows < M), which the panel's contraction then reads as it
  // would the decoded operand.
  __nv_bfloat16* a_out;
  long long lda_out;
};

struct Events {
  cudaEvent_t a, b;
  int stage;
};

// Arguments of one block scan (the tg_scan_block call).
struct ScanArgs {
  const uint8_t* G;
  int64_t ldg;
  int encoding;
  int64_t N, M, marker_offset;
  const uint32_t* missing;
  int64_t ldm;
  tg_scan_opts opts;
  tg_outputs out;
};

// Kernel choice per block-size bucket (floor(log2 M)), set by tg_autotune.
enum { TUNE_DEFAULT = 0, TUNE_PAIR = 1, TUNE_SINGLE = 2 };
constexpr int kTuneBuckets = 40;
inline int tune_bucket(int64_t M) {
  int b = 0;
  while ((M >> (b + 1)) > 0 && b + 1 < kTuneBuckets) ++b;
  return b;
}

}  // namespace tg

struct tg_panel {
  int device = 0;
  int64_t N = 0, P = 0, n_cov = 0, q = 0, df = 0, Npad = 0, Ppad = 0;
  int64_t NS = 0;               // samples the panel's phenotypes use (N unless a subset)
  uint32_t* samples = nullptr;  // [ceil(N/32)] bit mask of those samples (subset panels only)
  double* X = nullptr;        // [(1+n_cov)][N] design, reduced in place by the QR
  double* Q = nullptr;        // [q][N] (column-major N x q)
  double* Yres = nullptr;     // [P][N]
  double* s = nullptr;        // [P]
  float* col_s = nullptr;     // [P]
  float* col_rmul = nullptr;  // [Ppad]
  float* col_cs = nullptr;    // [Ppad] sum_i (Bhi + Blo)[p][i], in FP32
  __nv_bfloat16* Bhi = nullptr;  // [Ppad][Npad] unit-norm panel, high part
  __nv_bfloat16* Blo = nullptr;  // [Ppad][Npad] low part
  float* B32 = nullptr;          // [Ppad][Npad] unit-norm panel in FP32
  float* QB = nullptr;           // [QCOLS][Npad] Q columns 1..q-1 in FP32 (rest zero)
  __nv_bfloat16* QBhi = nullptr; // [QCOLS][Npad] the same split into bf16 hi + lo
  __nv_bfloat16* QBlo = nullptr;
  float* qcs = nullptr;          // [QCOLS] sum_i (QBhi + QBlo)[k][i]
  double lnB = 0;                // ln B(df/2, 1/2), df = N - q - 1
  double lnB_paper = 0;          // ln B((N-2)/2, 1/2) for the paper's printed form
  CUtensorMap tmBhi, tmBlo;      // phenotype panel, 256-row boxes
  CUtensorMap tmBhi2, tmBlo2;    // phenotype panel, 128-row boxes (one CTA's half of a pair tile)
  CUtensorMap tmQhi, tmQlo;      // covariate projection columns, 64-row boxes
  CUtensorMap tmBhi64, tmBlo64;  // phenotype panel, 64-row boxes (64-column tiles, P <= 64)
  // Small panels (P + q - 1 <= 256): the projection columns and the phenotypes in one operand
  // of joint_cols = 64, 128 or 256 rows, rows [0, q-1) = QB rows, rows [q-1, q-1+P) = the panel, rest
  // zero, so that one pass over a block's operand gives both Q^T a and the panel's products
  // (joint_cols = 0 and NULL buffers when the panel is larger).
  int joint_cols = 0;
  __nv_bfloat16* QYhi = nullptr;  // [joint_cols][Npad]
  __nv_bfloat16* QYlo = nullptr;
  float* qycs = nullptr;          // [joint_cols] qcs then col_cs
  CUtensorMap tmQYhi, tmQYlo;     // boxes of joint_cols rows
  // The same joint operand as f16 hi + lo of 2^14 v (joint_cols <= 128 only), for the joint pass
  // that decodes dosage rows in shared memory into f16 (k_fused.cu); scaled column sums.
  __half* QYhi16 = nullptr;       // [joint_cols][Npad]
  __half* QYlo16 = nullptr;
  float* qycs16 = nullptr;        // [joint_cols]
  CUtensorMap tmQYhi16, tmQYlo16;
  // The projection columns alone in the same f16 form (64 rows; panels with P + q - 1 > 128),
  // for the projection pass over dosage rows that also writes the block's operand (k_fused.cu).
  __half* QBhi16 = nullptr;       // [QCOLS][Npad]
  __half* QBlo16 = nullptr;
  float* qcs16 = nullptr;         // [QCOLS]
  CUtensorMap tmQhi16, tmQlo16;
  // The FP4 form's E2M1 pieces (built on the panel's first FP4 scan): the panel's columns
  // [kFp4Pieces][Ppad][Npad/2] and the projection columns [kFp4Pieces][QCOLS][Npad/2], each with
  // its column scale 2^-e (NaN: no test) and scaled column sum.
  uint8_t* fp4B = nullptr;
  float* fp4B_scale = nullptr;
  float* fp4B_cs = nullptr;
  uint8_t* fp4Q = nullptr;
  float* fp4Q_scale = nullptr;
  float* fp4Q_cs = nullptr;
  CUtensorMap tmFB, tmFQ;
};

struct tg_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t side = nullptr;
  uint32_t* status = nullptr;   // device word (ST_* bits)
  uint32_t* scratch = nullptr;  // small device scratch (rank, flags)
  // decode / projection workspace
  int64_t cap_rows = 0, cap_npad = 0;          // A buffers: rows x npad
  __nv_bfloat16* Ahi = nullptr;                 // centred split operand
  uint8_t* Afp4 = nullptr;                      // E2M1 operand of the FP4 form
  int64_t cap_fp4 = 0;                          // its bytes
  float* A32 = nullptr;
  int64_t cap_m = 0;                            // per-marker arrays
  int32_t* nobs = nullptr;
  double* mean = nullptr;
  float* shift = nullptr;                       // [cap_m] per-row shift of the split operand
  double* gc2s = nullptr;                       // [cap_m] |g_c|^2 over a subset panel's samples
  uint32_t* mh = nullptr;                       // [cap_m] bf16 bits of the missing-call value
  double* gc2 = nullptr;
  float* qg = nullptr;                          // [cap_m][QCOLS]
  double* gres2 = nullptr;
  float* rinv = nullptr;
  double* rinv64 = nullptr;
  int* refine_list = nullptr;                   // [cap_m] markers re-projected in FP64
  // host-streamed scan: a device ring of host_bufs block buffers' bytes (stage_cap allocated)
  uint8_t* stage = nullptr;
  size_t stage_cap = 0;
  int host_bufs = 3;
  tg_hit* dhits = nullptr;
  int64_t dhits_cap = 0;
  unsigned long long* dnhits = nullptr;
  unsigned long long* dbest = nullptr;
  int64_t dbest_cap = 0;
  cudaEvent_t ev_copied = nullptr;
  cudaEvent_t ev_free[tg::kRingEvents] = {};
  // timing of one block's copy (0, 1) and scan (2, 3) in a host-streamed scan, and their ratio
  // (scan time / copy time, 0 = not measured yet), which sets the next call's block ramp
  cudaEvent_t ev_rate[4 * tg::kRateBlocks] = {};
  double ramp_ratio = 0.0;
  double ramp_fixed = 0.0;  // > 0: a fixed growth factor set by the caller
  // profiling
  bool prof = false;
  std::vector<tg::Events> pending;
  std::vector<cudaEvent_t> event_pool;
  double stage_ms[TG_N_STAGES] = {0, 0, 0, 0, 0, 0};
  int64_t launches[TG_N_STAGES] = {0, 0, 0, 0, 0, 0};
  // captured scan graphs that hold pointers into this workspace
  int graphs_alive = 0;
  // split-form scans decode 2-bit / unmasked dosage blocks in the contraction producer
  // (off by default: slower than the decoded operand on GB300, see tg_set_fused_decode)
  bool fuse_decode = false;
  // small panels' joint projection pass reads the packed rows and decodes them in shared memory
  // (on by default: it removes the decoded operand's round trip through HBM)
  bool fuse_joint = true;
  // autotuned kernel per block-size bucket
  int tune_kernel[tg::kTuneBuckets] = {};
  int tune_group[tg::kTuneBuckets] = {};
  int tune_split[tg::kTuneBuckets] = {};        // split-K of the one-CTA kernel (0 = none)
  float* sk_ws = nullptr;                       // split-K partial sums and per-tile counters
  size_t sk_ws_bytes = 0;
  unsigned* sk_cnt = nullptr;
  int64_t sk_cnt_cap = 0;
};

namespace tg {

// error reporting and orchestration (api.cu)
tg_status fail(tg_status s, const std::string& msg);
tg_status cuda_fail(cudaError_t e, const char* what);
tg_status check_scan_args(const tg_ctx* c, const tg_panel* p, const ScanArgs& a);
tg_status scan_impl(tg_ctx* c, const tg_panel* p, const ScanArgs& a, cudaStream_t st);
// Degrees of freedom and ln B(df/2, 1/2) of the statistic a scan mode computes.
void mode_df(const tg_panel* p, int mode, double* df, double* lnB);
bool make_tmap(CUtensorMap* m, const void* ptr, int64_t rows, int64_t K, int64_t ld,
               uint32_t box_rows);
// uint8 map over packed genotype rows [rows][ld], boxes of box_bytes x box_rows, zero fill;
// swizzle64: the 64-byte swizzle (box_bytes must be 64).
bool make_tmap_packed(CUtensorMap* m, const void* ptr, int64_t rows, int64_t ld, uint32_t box_bytes,
                      uint32_t box_rows = 128, bool swizzle64 = false);

// panel kernels (k_panel.cu)
cudaError_t launch_build_design(double* X, const double* C, int64_t ldc, int64_t N, int64_t n_cov,
                                uint32_t* flags, cudaStream_t st);
cudaError_t launch_householder(double* X, int64_t N, int64_t k, double* Q, int* rank_out,
                               int* kept_out, cudaStream_t st);
cudaError_t launch_residualise(const float* Y, int64_t ldy, const double* Q, int64_t N, int64_t P,
                               int64_t q, int64_t Npad, double* Yres, double* s, float* col_s,
                               float* col_rmul, __nv_bfloat16* Bhi, __nv_bfloat16* Blo, float* B32,
                               float* col_cs, uint32_t* flags, cudaStream_t st);
// The joint operand of a small panel as scaled f16 hi + lo (rows of the q - 1 projection columns,
// then the P phenotypes, zero to `rows`), with its scaled column sums.
cudaError_t launch_joint_f16(const double* Q, int64_t N, int64_t nq, const double* Yres,
                             const double* s, const float* rmul, int64_t P, int64_t rows,
                             int64_t Npad, __half* hi, __half* lo, float* cs, cudaStream_t st);
cudaError_t launch_qcols(const double* Q, int64_t N, int64_t q, int64_t Npad, float* QB,
                         __nv_bfloat16* QBhi, __nv_bfloat16* QBlo, float* qcs, cudaStream_t st);
// subset panels: rows gathered to a compact copy and scattered back (elements of 2, 4 or 8
// bytes), and per-phenotype finite-value masks
cudaError_t launch_gather_f32(const float* src, int64_t lds, float* dst, int64_t ldd, const int* idx,
                              int64_t ns, int64_t R, cudaStream_t st);
cudaError_t launch_gather_f64(const double* src, int64_t lds, double* dst, int64_t ldd,
                              const int* idx, int64_t ns, int64_t R, cudaStream_t st);
cudaError_t launch_scatter(const void* src, int64_t lds, void* dst, int64_t ldd, const int* idx,
                           int64_t ns, int64_t R, int elem_bytes, cudaStream_t st);
cudaError_t launch_pheno_masks(const float* Y, int64_t ldy, int64_t N, int64_t P, uint32_t* masks,
                               int64_t ldm, cudaStream_t st);

// decode (k_decode.cu)
cudaError_t launch_decode(const uint8_t* G, int64_t ldg, int encoding, int64_t N, int64_t M,
                          const uint32_t* missing, int64_t ldm, int precision, void* Ahi,
                          float* shift, uint32_t* mh, int64_t lda, int32_t* nobs, int64_t* S,
                          int64_t* S2, double* mean, double* gc2, cudaStream_t st);
// |g_c|^2 over the samples of a subset panel (decode units; the imputed value is the marker's
// all-sample mean)
cudaError_t launch_subset_stats(const uint8_t* G, int64_t ldg, int encoding, int64_t N, int64_t M,
                                const uint32_t* missing, int64_t ldm, const uint32_t* samples,
                                const double* mean, double* gc2s, cudaStream_t st);

// SIMT kernels (k_simt.cu)
cudaError_t launch_project(const float* A, int64_t lda, int64_t M, int64_t K, const float* QB,
                           int64_t nq, float* qg, cudaStream_t st);
// What the FP64 re-projection of markers close to the covariate span needs: the packed block,
// the FP64 means (units) and the panel's FP64 basis Q ([q][N], column 0 the intercept), and a
// list of at least M ints with its counter (4 bytes of device memory).
struct MarkerRefine {
  const uint8_t* G;
  int64_t ldg;
  int encoding;
  int64_t N;
  const uint32_t* missing;
  int64_t ldm;
  const double* mean;
  const double* Q;
  int q;
  int* list;
  unsigned* count;
};
// complete_n > 0: markers with fewer than complete_n observed calls are untestable too.
cudaError_t launch_marker_norm(int64_t M, const int32_t* nobs, const double* gc2, const float* qg,
                               int64_t ldq, int64_t nq, double kappa, double* gres2_units_out,
                               double* norm2_allele_out, float* rinv, double* rinv64,
                               const MarkerRefine* refine, cudaStream_t st, int64_t complete_n = 0);
cudaError_t launch_sgemm_scan(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t K,
                              const EpiParams& ep, cudaStream_t st);

// statistics after the contraction (k_stats.cu)
cudaError_t launch_full_stats(const EpiParams& ep, cudaStream_t st);
cudaError_t launch_hit_stats(const EpiParams& ep, const unsigned long long* start, cudaStream_t st);
cudaError_t launch_fill_random(uint8_t* p, size_t n, unsigned long long seed, cudaStream_t st);

// tensor-core kernel (k_tc.cu)
// With `dec` non-NULL the A operand is decoded from packed genotypes in the kernel (tmA unused).
// `narrow`: 64-column tiles for a panel of at most 64 phenotypes (B maps with 64-row boxes).
// Raw mode (ep.raw_out: the covariate projection, alone or joint with a small panel) uses the
// narrowest of 64-, 128- and 256-column tiles that holds the raw columns.
cudaError_t launch_tc_scan(const CUtensorMap* tmA, const CUtensorMap* tmBhi,
                           const CUtensorMap* tmBlo, int64_t K, const EpiParams& ep, int sm_count,
                           long long spin_ns, cudaStream_t st, int group_m = 16,
                           const DecodeArgs* dec = nullptr, int encoding = 0, bool narrow = false);

// The joint projection pass of a small panel (joint operand of 64 or 128 rows) with the decode
// fused in (k_fused.cu): reads the packed rows through da.tmG, whose boxes must be
// joint_fused_rows(M, sm_count, joint_cols) rows of 64 bytes with the 64-byte swizzle (dosage)
// or 16 bytes (2-bit calls); raw mode only, no split-K, K a multiple of 64. Writes the raw
// products launch_tc_scan writes.
int joint_fused_rows(int64_t M, int sm_count, int joint_cols);
// Dosage rows are expanded into f16 (b - c exact) against the f16 joint operand (tmBhi / tmBlo
// then map QYhi16 / QYlo16 and ep.col_cs is qycs16; the raw products are scaled back by 2^-14);
// 2-bit calls into bf16 against the bf16 joint operand.
cudaError_t launch_joint_fused(const CUtensorMap* tmBhi, const CUtensorMap* tmBlo, int64_t K,
                               const EpiParams& ep, int sm_count, long long spin_ns, cudaStream_t st,
                               const DecodeArgs& da, int encoding);

// The statistics of a small panel (P <= 256) from the joint pass's raw products (k_tc.cu): D of
// marker row m and phenotype p at raw[m * ld + p] (the shift's add-back included), the same
// per-element epilogue as the contraction kernels.
cudaError_t launch_raw_stats(const float* raw, int64_t ld, const EpiParams& ep, cudaStream_t st);

// The FP4 form (k_fp4.cu). Pieces: rows r < nrows of src (stride lds; divided by div[r] when
// div is not NULL; skipped where valid[r] is NaN) as kFp4Pieces E2M1 pieces, out[k][rows_pad][Npad/2]
// bytes, with scale[r] = 2^-e (NaN for a skipped row) and cs[r] = the scaled column sum.
cudaError_t launch_fp4_pieces(const double* src, int64_t lds, const double* div, const float* valid,
                              int64_t nrows, int64_t rows_pad, int64_t N, int64_t Npad, uint8_t* out,
                              float* scale, float* cs, cudaStream_t st);
// The FP4 form's decode of 2-bit rows in one pass: the E2M1 operand [M][lda] bytes (lda =
// Npad / 2, a multiple of 32) and each row's n_obs, FP64 mean, |g_c|^2 and shift = -mean.
cudaError_t launch_fp4_decode(const uint8_t* G, int64_t ldg, int64_t N, int64_t M, uint8_t* A,
                              int64_t lda, int32_t* nobs, double* mean, double* gc2, float* shift,
                              cudaStream_t st);
// The contraction: tmA over the E2M1 operand (boxes of 64 bytes x 128 rows, 64-byte swizzle),
// tmB over kFp4Pieces x b_rows_pad piece rows (boxes of 64 bytes x 128 rows, or 64 rows in raw
// mode: the covariate projection, at most 64 columns).
cudaError_t launch_fp4_scan(const CUtensorMap* tmA, const CUtensorMap* tmB, int b_rows_pad,
                            int64_t Npad, const EpiParams& ep, int sm_count, long long spin_ns,
                            cudaStream_t st);

// tensor-core kernel on CTA pairs, 256 x 256 tiles (k_tc2.cu)
cudaError_t launch_tc2_scan(const CUtensorMap* tmA, const CUtensorMap* tmBhi,
                            const CUtensorMap* tmBlo, int64_t K, const EpiParams& ep, int sm_count,
                            long long spin_ns, cudaStream_t st, int group_m = 16,
                            const DecodeArgs* dec = nullptr, int encoding = 0);

// bounded wait test (k_tc.cu)
cudaError_t launch_wait_test(const uint32_t* flag, long long limit_ns, uint32_t* result,
                             cudaStream_t st);

// p-value helpers on the host (pvalue.cuh)
double host_lnbeta_half(double df);
double host_r2_threshold(double mlog10p, double df, double lnB);

}  // namespace tg
