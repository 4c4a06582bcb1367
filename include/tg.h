/*
 * tg.h - C ABI of the GB300 genome-scan library (libtg.so).
 *
 * Method: TorchGWAS (arXiv 2604.21095), Section 2.2. A phenotype panel Y (N samples x P
 * traits) is mean-centred, residualised against an orthonormal covariate basis Q and
 * standardised once (Eq. 1); each block of M markers is then decoded, standardised and
 * correlated with the whole panel (Eq. 2), and every correlation is turned into a t
 * statistic (Eq. 3), a -log10 p-value, an effect size and its standard error.
 *
 * Conventions for every call:
 *   - Data pointers marked "device" are CUDA device memory owned by the caller; the
 *     library never frees them. Pointers marked "host" are host memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *     asynchronous on it unless stated otherwise; argument errors are returned
 *     synchronously, before any work is queued.
 *   - Errors found by a kernel (hit-buffer overflow, a bounded wait that ran out) are
 *     latched in a per-context device status word and returned by tg_status_poll().
 *   - On failure a call returns a non-zero tg_status and sets a thread-local message
 *     readable with tg_last_error().
 *   - Matrices are dense with an explicit leading dimension (elements unless noted).
 *   - Only sm_103a (GB300) is supported; every compute step runs in the library's own
 *     CUDA kernels. There is no CPU path.
 */
#ifndef TG_H_
#define TG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TG_ABI_VERSION 2

typedef struct tg_ctx tg_ctx;
typedef struct tg_panel tg_panel;

typedef enum {
  TG_OK = 0,
  TG_ERR_INVALID_ARG = 1, /* bad pointer, size, stride, alignment or enum */
  TG_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  TG_ERR_OOM = 3,         /* device allocation failed */
  TG_ERR_NONFINITE = 4,   /* NaN or Inf in the phenotypes or covariates */
  TG_ERR_RANK = 5,        /* too few samples for the covariate rank (N <= q + 1) */
  TG_ERR_CAPACITY = 6,    /* more hits than the hit buffer holds (the count is still exact) */
  TG_ERR_TIMEOUT = 7,     /* a bounded device-side wait ran out */
  TG_ERR_UNSUPPORTED = 8  /* a size beyond the library's limits, or no sm_103a device */
} tg_status;

typedef enum {
  TG_PREC_FP32 = 0,       /* FP32 operands, FP32 SIMT contraction */
  TG_PREC_SPLIT_BF16 = 1, /* exact BF16 genotype codes, panel split into BF16 hi + lo,
                             two tcgen05 tensor-core products accumulated in FP32 */
  TG_PREC_FP4_PIECES = 2  /* experimental, 2-bit calls only: exact E2M1 genotype counts, each
                             panel column scaled by a power of two and split into 6 E2M1 pieces
                             (piece k at scale 8^-k), block-scaled tcgen05 kind::mxf4 products
                             accumulated in FP32. A marker with a missing call has no test in this
                             form (NaN outputs, no hit): the E2M1 operand cannot hold its imputed
                             mean. The pieces of a panel (6 x round_up(P, 256) x round_up(N, 64) / 2
                             bytes) are built on its first FP4 scan, synchronously. Dosage blocks,
                             subset panels, tg_scan_block_static and captured graphs give
                             TG_ERR_UNSUPPORTED. */
} tg_precision;

typedef enum {
  TG_ENC_2BIT = 0,     /* PLINK 1 .bed SNP-major: sample i in bits 2(i%4)+{0,1} of byte i/4;
                          field 00 -> 2 copies of allele 1, 10 -> 1, 11 -> 0, 01 -> missing */
  TG_ENC_U8_DOSAGE = 1 /* one byte b per sample, allele-1 dosage 2b/255 */
} tg_encoding;

/* Which statistic the scan computes (Section 2.2). */
typedef enum {
  TG_MODE_PROJECTED = 0, /* the OLS test of y on [1, C, g]: the marker is projected on Q as well,
                            r = g_res.y_res / (|g_res| |y_res|), df = N - q - 1 */
  TG_MODE_PAPER = 1      /* Eq. 2-3 as printed: the marker is only centred and standardised,
                            r = g_c.y_res / (|g_c| |y_res|), df = N - 2 whatever the covariates
                            (identical to TG_MODE_PROJECTED when the covariates are an intercept
                            only); beta = g_c.y_res / |g_c|^2, se = |beta / t| */
} tg_mode;

/* Per-call scan options. */
typedef struct {
  int32_t precision;   /* tg_precision */
  int32_t full_output; /* nonzero: write beta, se, t, -log10 p of every (marker, phenotype) */
  double hit_mlog10p;  /* collect pairs with -log10 p >= this; <= 0 or NaN: no hit list */
  int32_t mode;        /* tg_mode (0 = TG_MODE_PROJECTED) */
  int32_t reserved;    /* must be 0 */
} tg_scan_opts;

/* One association above the hit threshold (24 bytes). */
typedef struct {
  uint32_t marker; /* marker_offset + row within the block */
  uint32_t pheno;  /* phenotype column */
  float beta;      /* OLS effect of one allele-1 copy */
  float se;        /* its standard error */
  float t;         /* Eq. 3 t statistic, df = N - q - 1 */
  float mlog10p;   /* -log10 of the two-sided p-value */
} tg_hit;

/* Outputs of tg_scan_block. Every pointer is device memory and may be NULL when that
 * output is not wanted (beta/se/t/mlog10p are ignored unless opts->full_output). */
typedef struct {
  float* beta;    /* [M][ldo] row-major: row = marker of the block, column = phenotype */
  float* se;
  float* t;
  float* mlog10p;
  int64_t ldo;            /* >= P */
  tg_hit* hits;           /* hit records, unordered; [hit_capacity] */
  int64_t hit_capacity;
  unsigned long long* n_hits; /* running count; the caller zeroes it. Counts every hit, also
                                 those past hit_capacity (then TG_ERR_CAPACITY is latched) */
  unsigned long long* best;   /* [P] running per-phenotype best marker; the caller zeroes it.
                                 key = (bits of float |r|) << 32 | (0xFFFFFFFF - marker):
                                 larger |r| wins, ties go to the smaller marker */
  double* marker_norm2;   /* [M] |g_res|^2 in allele units (NaN: marker untestable: no observed
                             call, constant, or in TG_MODE_PROJECTED a variance inflation
                             factor |g_c|^2 / |g_res|^2 above 50 on the covariates) */
  int32_t* marker_nobs;   /* [M] observed calls */
  double* marker_mean;    /* [M] observed mean in decode units (counts, or bytes for dosages) */
} tg_outputs;

/* Library version string and ABI number. */
const char* tg_version(void);
int tg_abi_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* tg_last_error(void);
const char* tg_status_string(tg_status s);

/* Create a context on CUDA device `device`: workspace, status word, side stream.
 * Fails with TG_ERR_UNSUPPORTED unless the device is sm_103. */
tg_status tg_create(tg_ctx** ctx, int device);
tg_status tg_destroy(tg_ctx* ctx);

/* Section 2.2, Eq. 1 and the standardisation after it.
 * Builds X = [1, C], an orthonormal basis Q of span(X) by FP64 Householder QR (a column
 * whose remaining norm is <= 1e-9 of its own norm is dropped; q = rank), the residualised
 * panel Y_res = (I - Q Q^T)(Y - Ybar) in FP64, the column norms s_p = |y_res,p| and the
 * unit-norm panel in the forms the scan consumes. A panel with P + q - 1 <= 256 also keeps a
 * joint copy of its split operand behind the q - 1 projection columns (64, 128 or 256 rows of
 * round_up(N, 64) bf16 pairs), so that split-form scans in the projected mode take the
 * projection and the panel's products from one pass over each block.
 *   Y: device, float [P][ldy] storage = column-major N x P (phenotype p at Y + p*ldy), ldy >= N.
 *   C: device, double column-major N x n_cov (covariate k at C + k*ldc), ldc >= N; NULL if n_cov = 0.
 *      The intercept is added by the library and must not be passed.
 * Synchronous: returns after the panel is ready. A phenotype whose residual norm is
 * <= 1e-12 of its centred norm has no test (its outputs are NaN).
 * Errors: TG_ERR_NONFINITE (NaN/Inf in Y or C), TG_ERR_RANK (N <= q + 1),
 * TG_ERR_UNSUPPORTED (n_cov > 63), TG_ERR_INVALID_ARG. The panel is owned by the library. */
tg_status tg_prepare_panel(tg_ctx* ctx, const float* Y, int64_t ldy, int64_t N, int64_t P,
                           const double* C, int64_t ldc, int64_t n_cov, tg_panel** out,
                           void* stream);

/* Panel shape: samples, phenotypes, covariate rank q (intercept included), df = N - q - 1. */
/* The panel of a group of phenotypes observed on a subset S of the N samples (phenotypes that
 * share one missingness pattern; the paper has no missing phenotypes, this is the reading
 * taken for them). Eq. 1 and the standardisation are applied to the rows in S only, with
 * X = [1, C] restricted to S, and every scan of the panel tests the OLS of y_S on
 * [1, C_S, g_S] (or Eq. 2-3 on S in TG_MODE_PAPER), df = N_S - q - 1 (N_S - 2). A genotype's
 * missing calls are still imputed with its mean over all N samples.
 *   Y, ldy, N, P, C, ldc, n_cov: as tg_prepare_panel; phenotype values outside S are never
 *   read (NaN allowed there), inside S they must be finite.
 *   samples: device, uint32 [ceil(N/32)], bit i%32 of word i/32 set = sample i in S (bits
 *   past N ignored); N_S >= 3.
 * The panel keeps the full sample axis (its arrays are zero outside S), so blocks of all N
 * samples are scanned against it with tg_scan_block, tg_scan_host and the captured graphs;
 * tg_scan_block_static rejects it (TG_ERR_UNSUPPORTED). Subset panels concatenate only with
 * panels of the same subset. Synchronous. */
tg_status tg_prepare_panel_subset(tg_ctx* ctx, const float* Y, int64_t ldy, int64_t N, int64_t P,
                                  const double* C, int64_t ldc, int64_t n_cov,
                                  const uint32_t* samples, tg_panel** out, void* stream);

/* The samples a panel uses: n_used = N_S (N for a panel of all samples) and a borrowed device
 * pointer to its sample mask (NULL for a panel of all samples). */
tg_status tg_panel_samples(const tg_panel* panel, int64_t* n_used, const uint32_t** samples);

/* Per-phenotype masks of finite values, the input for grouping phenotypes by missingness:
 * masks[p * ldm + w] bit b set = Y[p * ldy + 32 w + b] is finite (bits past N are 0).
 * Y: device float [P][ldy]; masks: device uint32 [P][ldm], ldm >= ceil(N/32). Asynchronous. */
tg_status tg_phenotype_masks(tg_ctx* ctx, const float* Y, int64_t ldy, int64_t N, int64_t P,
                             uint32_t* masks, int64_t ldm, void* stream);

tg_status tg_panel_info(const tg_panel* panel, int64_t* N, int64_t* P, int64_t* q, int64_t* df);

/* Borrowed device pointer to Q: double column-major N x q (column k at Q + k*ldq). */
tg_status tg_panel_Q(const tg_panel* panel, const double** Q, int64_t* ldq, int64_t* q);

/* Borrowed device pointers to Y_res (double column-major N x P, column p at Yres + p*ld)
 * and to s (double [P], column norms of Y_res). */
tg_status tg_panel_Yres(const tg_panel* panel, const double** Yres, int64_t* ld, const double** s);

tg_status tg_panel_free(tg_panel* panel);

/* Section 2.2, genotype batches: decode one block of M markers into the contraction
 * operand and the exact per-marker statistics (the first step of tg_scan_block, exposed
 * on its own for testing and for callers that keep the operand).
 *   G: device, uint8 [M][ldg]; ldg >= ceil(N/4) (2-bit) or >= N (dosage), ldg % 16 == 0,
 *      G 16-byte aligned.
 *   missing: device, uint32 [M][ldm] bit mask (bit i%32 of word i/32 set = call i missing),
 *      ldm >= ceil(N/32); dosage only (must be NULL for 2-bit, where it is in-band); may be NULL.
 *   A: device operand rows of lda elements, lda >= N, lda % 64 == 0, 16-byte aligned;
 *      columns N..lda-1 are written 0.
 *      TG_PREC_FP32: float; an observed call holds its code (or byte), a missing call
 *      float(mean).
 *      TG_PREC_SPLIT_BF16: bf16, the row centred on a shift c: c = round(128 mean) / 128 for
 *      2-bit calls, round(mean) for dosage bytes (round half to even; c = 0 if n_obs = 0), so
 *      that an observed call holds code - c exactly and a missing call bf16(mean - c)
 *      (|mean - c| <= 1/256 or 1/2). The scan adds c sum_i y_i back per phenotype.
 *   shift: device float [M], receives c (exact in float); split form only (NULL for FP32,
 *      where it must be NULL); may be NULL.
 *   n_obs, S, S2 (int32/int64/int64 [M]): exact observed count, sum and sum of squares in
 *      decode units; mean (double [M]): S / n_obs, one correctly rounded division (NaN if
 *      n_obs = 0). Any of these four may be NULL. */
tg_status tg_decode_block(tg_ctx* ctx, const uint8_t* G, int64_t ldg, int32_t encoding, int64_t N,
                          int64_t M, const uint32_t* missing, int64_t ldm, int32_t precision,
                          void* A, float* shift, int64_t lda, int32_t* n_obs, int64_t* S,
                          int64_t* S2, double* mean, void* stream);

/* Section 2.2 Eq. 2 and Eq. 3 for one block: decode (mean imputation of missing calls),
 * project each marker on Q (|g_res|^2 = |g_c|^2 - |Q^T g_c|^2), contract the block with the
 * whole panel, and turn every correlation r into t = r sqrt(df / (1 - r^2)),
 * beta = r s_p / |g_res|, se = |beta / t| and -log10 p, p = I_{1-r^2}(df/2, 1/2) (two-sided).
 * A marker with no observed call, a constant one, or (TG_MODE_PROJECTED) one whose variance
 * inflation factor on the covariates, |g_c|^2 / |g_res|^2, exceeds 50 (the covariates explain
 * more than 98% of its variance) is untestable: NaN outputs, no hit, never a best marker.
 *   G, ldg, encoding, missing, ldm: as tg_decode_block; N must equal the panel's N.
 *   marker_offset: global index of the block's first marker (used in hits and best).
 *   opts: precision, full output and hit threshold. out: see tg_outputs.
 * Workspace is grown on demand (cudaMalloc); a call with a larger M than any before may
 * therefore synchronise the device. M = 0 is a no-op. */
tg_status tg_scan_block(tg_ctx* ctx, const tg_panel* panel, const uint8_t* G, int64_t ldg,
                        int32_t encoding, int64_t N, int64_t M, int64_t marker_offset,
                        const uint32_t* missing, int64_t ldm, const tg_scan_opts* opts,
                        const tg_outputs* out, void* stream);

/* The same block scan for callers that cannot allocate device memory. The paper has no
 * counterpart: this is a deployment variant. Some callers must not call cudaMalloc or cudaFree
 * while they scan, e.g. a host application whose device memory belongs to another allocator
 * (a framework's caching pool, a fixed budget), or a latency-critical loop that cannot take
 * the device-wide synchronisation cudaMalloc/cudaFree may cause. This call needs no context
 * and allocates nothing: its scratch (decoded genotype operand, per-marker statistics, status
 * word) is one static device array of 64 MiB that every GPU loading the library keeps until
 * the process exits.
 *   Arguments and outputs: as tg_scan_block (the panel comes from tg_prepare_panel, made
 *   beforehand). The current device must be the panel's device.
 *   Limit: the block must fit the 64 MiB scratch, about (2 bytes split, 4 bytes FP32) x
 *   round_up(N, 64) per marker, e.g. about 1,400 markers at N = 23,000 or 15,000 at N = 2,000
 *   in the split form; larger blocks return TG_ERR_UNSUPPORTED with the maximum in the
 *   message, before anything is launched.
 *   The first call on a device does a one-time set-up (it looks up the array's device address
 *   with cudaGetSymbolAddress while that device is current); make that first call before any
 *   stream capture.
 *   Every call shares the one array, which keeps the last call's contents (the call clears
 *   what must start at zero): calls that overlap on the GPU, from several threads or streams,
 *   race on it and must be serialised by the caller.
 *   Synchronous: returns after the scan finished on `stream`, with TG_ERR_CAPACITY or
 *   TG_ERR_TIMEOUT if the kernels reported one. */
tg_status tg_scan_block_static(const tg_panel* panel, const uint8_t* G, int64_t ldg,
                               int32_t encoding, int64_t N, int64_t M, int64_t marker_offset,
                               const uint32_t* missing, int64_t ldm, const tg_scan_opts* opts,
                               const tg_outputs* out, void* stream);

/* The scan of a whole genotype matrix held in HOST memory (pinned for overlap): blocks of
 * at most block_markers rows are copied to the device on the context's side stream, into a
 * device ring the size of a few full blocks (3 by default, tg_set_host_buffers), while earlier
 * blocks are scanned on `stream`; hits, their count and the per-phenotype best keys are copied
 * back to host memory at the end. Synchronous.
 *   The ring: blocks are placed back to back (each on a 256-byte boundary) and wrap to its
 *   start; a copy waits only for the scans of the blocks whose bytes it overwrites, so the
 *   smaller ramped blocks let the copies run up to 8 x n_buffers blocks ahead.
 *   Blocking: when block_markers >= 2048 the first block has round_up(block_markers / 8, 256)
 *   rows and each next block f times as many (rounded up to 256), up to block_markers, so that
 *   only a short first copy is not hidden behind a scan. f = 2 on a context's first host scan;
 *   each call times the copies and scans of its second to ninth blocks, and later calls use
 *   the ratio of their sums (scan / copy) clamped to [1, 2], so that a slow host link keeps the
 *   blocks small instead of leaving the scan waiting on a copy twice its own length. Results do
 *   not depend on the blocking.
 *   G_host: host uint8 [M][ldg]; hits_host: host [hit_capacity]; n_hits: host, total hit
 *   count (may exceed hit_capacity, then TG_ERR_CAPACITY); best_host: host [P] or NULL.
 *   Like tg_status_poll, the call reads and clears the context's device status word at the
 *   end: TG_ERR_TIMEOUT if a bounded device wait ran out, TG_ERR_CAPACITY on overflow.
 * Only hit collection is supported here (opts->full_output must be 0). */
tg_status tg_scan_host(tg_ctx* ctx, const tg_panel* panel, const uint8_t* G_host, int64_t ldg,
                       int32_t encoding, int64_t N, int64_t M, int64_t block_markers,
                       int64_t marker_offset, const tg_scan_opts* opts, tg_hit* hits_host,
                       int64_t hit_capacity, int64_t* n_hits, unsigned long long* best_host,
                       void* stream);

/* The block growth factor f of tg_scan_host: factor = 0 (the default) picks it from the
 * previous call's measured scan / copy ratio as described there; 1 <= factor <= 8 fixes it.
 * TG_ERR_INVALID_ARG for other values. */
tg_status tg_set_host_ramp(tg_ctx* ctx, double factor);

/* The size of tg_scan_host's device ring in full blocks (2, 3 or 4; 3 on a new context):
 * n_buffers x block_markers x ldg bytes (each block rounded up to 256 bytes) of device memory,
 * allocated by the next call. With two and full-size blocks, a block's copy waits for the scan
 * of the block two before it, so any copy slower than the scan it runs beside stalls the scan;
 * each further full block of ring lets the copies run one more block ahead, which absorbs a host
 * link whose rate varies from copy to copy as long as its average keeps up. Ramped blocks are
 * smaller, so more of them fit. TG_ERR_INVALID_ARG for other values. */
tg_status tg_set_host_buffers(tg_ctx* ctx, int n_buffers);

/* The factor the next tg_scan_host call will use, and the last measured scan / copy time ratio
 * of one block (0 before any measurement). Either pointer may be NULL. */
tg_status tg_host_ramp(const tg_ctx* ctx, double* factor, double* measured_ratio);

/* The block sizes tg_scan_host uses for M markers, blocks of at most block_markers and growth
 * factor `factor` in [1, 8] (host only, no device work): *n_blocks = their number, and the
 * first min(capacity, *n_blocks) sizes are written to `sizes` (host int64 [capacity]; NULL
 * with capacity 0 returns the count alone, with no list built). block_markers is at most 2^32
 * (TG_ERR_INVALID_ARG above, here and in tg_scan_host). TG_ERR_UNSUPPORTED when M would take
 * 2^28 blocks or more. */
tg_status tg_host_block_sizes(int64_t M, int64_t block_markers, double factor, int64_t* sizes,
                              int64_t capacity, int64_t* n_blocks);

/* Where split-form scans decode the genotypes inside the contraction kernels instead of first
 * writing the decoded operand (about 2 x round_up(N, 64) bytes per marker) to device memory.
 * The fused forms apply to 2-bit blocks and to dosage blocks without a missing mask (others always
 * use the decoded operand). They compute bit-identical results, except the small-panel pass on
 * dosage blocks (enable = 2 or 1), which expands the bytes into f16 (b - c exactly) against an
 * f16 hi + lo copy of the joint operand (about 22 significant bits against bf16's 16): its
 * results differ from the decoded operand's within the float tolerance.
 *   enable = 2 (the default): only the joint projection pass of a small panel (projected mode,
 *     P + q - 1 <= 128, blocks of at least one 128-marker tile per SM), where the scan is one pass
 *     bound by the bytes it reads: the pass reads the packed rows (1 or 1/4 byte per sample)
 *     and decodes them on chip with 8 decoder warps, removing the operand's write and read
 *     (Section 2.4: the scan is bound by the reader's bandwidth). A counting pass over the rows
 *     (n_obs, sums, the mean each row is centred on) comes first, except for dosage rows on
 *     256-marker tiles (blocks of at least 256 markers per SM, N <= 66,051): there the pass
 *     centres each row on the rounded mean of its first 64 bytes and takes the row's exact
 *     sums as it expands it, so the block is read once. The statistics are the same integers
 *     and the same FP64 mean either way.
 *   The same setting runs a larger panel's projection (P + q - 1 > 128; same conditions
 *     otherwise) as that pass with the q - 1 projection columns alone, which also writes the
 *     block's decoded operand as it expands the rows (the contraction of the panel then reads
 *     it): the operand is written once and read once instead of read a second time for the
 *     projection. Dosage rows take f16 projection columns there and, on 256-marker tiles, the
 *     one-pass statistics above; 2-bit calls give results bit-identical to enable = 0 for
 *     panels with P + q - 1 > 256.
 *   enable = 1: also the contraction kernels of larger panels, whose two decoder warps per CTA
 *     take about 3,000 cycles per 32-sample K block against 512 for the products, so on GB300
 *     they are slower there.
 *   enable = 0: never; every block goes through the decoded operand.
 * Not allowed while a captured scan graph uses the context (TG_ERR_INVALID_ARG); other values
 * give TG_ERR_INVALID_ARG. */
tg_status tg_set_fused_decode(tg_ctx* ctx, int enable);

/* ---- Batched form: many panels, ragged blocks, one captured graph, tuned tiles ----------- */

/* One panel made of n panels that were prepared from the same N samples and the same
 * covariates (their covariate bases must be bit-identical; otherwise TG_ERR_INVALID_ARG):
 * the phenotype columns are concatenated in order, so panel i's columns start at the sum of
 * the earlier panels' P. Scanning it runs one persistent kernel over all panels' columns
 * (Section 2.1: the panel is prepared once and reused; here several panels share one scan).
 * The inputs stay valid and owned by the caller; the result is a new library-owned panel.
 * Synchronous. */
tg_status tg_panel_concat(tg_ctx* ctx, const tg_panel* const* panels, int n, tg_panel** out,
                          void* stream);

typedef struct tg_graph tg_graph;

/* Capture the scans of n_blocks genotype blocks (each as tg_scan_block: device pointer G[b],
 * M[b] markers, global marker offset marker_offset[b], optional mask missing[b]; the arrays
 * themselves are host memory) into one CUDA graph. Hits, their count and the per-phenotype
 * best keys accumulate in `out` over all blocks; full output and per-marker outputs are not
 * supported here. The context's workspace is sized for the largest block before the capture
 * and is then held by the graph: while the graph exists, tg_scan_block on the same context
 * only accepts blocks that fit it. */
tg_status tg_scan_graph_create(tg_ctx* ctx, const tg_panel* panel, int n_blocks,
                               const uint8_t* const* G, const int64_t* M,
                               const int64_t* marker_offset, const uint32_t* const* missing,
                               int64_t ldg, int64_t ldm, int32_t encoding, int64_t N,
                               const tg_scan_opts* opts, const tg_outputs* out, tg_graph** graph);
/* The same with the genotype blocks in host memory: G_host[b] holds M[b] rows of ldg bytes in
 * page-locked host memory (no missing masks: 2-bit calls carry theirs in-band, dosage blocks
 * are scanned unmasked). The graph owns two device staging buffers of the largest block; each
 * replay copies every block into one of them on a stream forked inside the graph, so that the
 * copy of block b+1 runs while block b is scanned (Section 2.2, batches streamed in), and
 * joins that stream before it ends. The host blocks are read at every replay: refill them
 * between replays to stream new markers through the same graph. Same output rules as
 * tg_scan_graph_create. */
tg_status tg_scan_graph_create_host(tg_ctx* ctx, const tg_panel* panel, int n_blocks,
                                    const uint8_t* const* G_host, const int64_t* M,
                                    const int64_t* marker_offset, int64_t ldg, int32_t encoding,
                                    int64_t N, const tg_scan_opts* opts, const tg_outputs* out,
                                    tg_graph** graph);
/* Replay the captured scans on `stream` (asynchronous). */
tg_status tg_scan_graph_launch(tg_graph* graph, void* stream);
tg_status tg_scan_graph_free(tg_graph* graph);

/* Time the tensor-core scan of an M-marker block of this panel with each candidate kernel
 * (CTA pairs on 256 x 256 tiles, or one CTA per 128 x 256 tile) and raster group, on a
 * pseudo-random block, and keep the fastest for blocks of this size (same power of two) in the
 * context. Synchronous; allocates a temporary block. */
tg_status tg_autotune(tg_ctx* ctx, const tg_panel* panel, int32_t encoding, int64_t M,
                      void* stream);
/* The tuned choice for M-marker blocks: kernel 2 = CTA pairs, 1 = one CTA per tile; group =
 * m-tiles per raster group. */
tg_status tg_tuning(const tg_ctx* ctx, int64_t M, int32_t* kernel, int32_t* group);
/* Set the choice for M-marker blocks by hand (e.g. from a saved tuning): kernel 1 or 2, group
 * in [1, 1024]. */
tg_status tg_set_tuning(tg_ctx* ctx, int64_t M, int32_t kernel, int32_t group);
/* Split-K of the one-CTA kernel for M-marker blocks of panels wider than 64 phenotypes: 1, 2
 * or 4 chunk-aligned ranges of the samples, whose partial sums the tile's first range adds in
 * order (so results do not depend on scheduling). tg_autotune tries 2 and 4 when that kernel's
 * tiles are fewer than half the SMs; panels of at most 64 phenotypes split by the same rule
 * without tuning. */
tg_status tg_set_tuning_split(tg_ctx* ctx, int64_t M, int32_t splits);
tg_status tg_tuning_split(const tg_ctx* ctx, int64_t M, int32_t* splits);
/* Keep a tuning: write every tuned block-size bucket of the context to a small JSON file
 * ({"format": "tg-tuning", "version": 1, "buckets": [{"min_markers", "kernel": "pair" or
 * "single", "group_m", "splits"}, ...]}), and read such a file into a context (a tuning taken
 * once on a GB300 reused by later runs). Loading checks every entry first and changes nothing
 * if one is malformed (TG_ERR_INVALID_ARG). Host file I/O only; synchronous. */
tg_status tg_tuning_save(const tg_ctx* ctx, const char* path);
tg_status tg_tuning_load(tg_ctx* ctx, const char* path);

/* Synchronise `stream`, then return and clear the latched device status
 * (TG_ERR_CAPACITY, TG_ERR_TIMEOUT) of work queued so far. */
tg_status tg_status_poll(tg_ctx* ctx, void* stream);

/* Stage timing with CUDA events on the launching stream (off by default). */
#define TG_N_STAGES 6 /* 0 decode, 1 projection, 2 marker norm, 3 contraction + epilogue,
                         4 H2D copies, 5 statistics of hits / full output */
tg_status tg_set_profiling(tg_ctx* ctx, int enable);
/* Total milliseconds and kernel launches per stage since the last reset (synchronises
 * the recorded events). Either array may be NULL. */
tg_status tg_stage_times(tg_ctx* ctx, double* ms, int64_t* launches, int reset);

/* Spin on a device word until it becomes nonzero or limit_ns elapses, with the same
 * bounded wait the scan kernels use. Returns TG_ERR_TIMEOUT (and latches nothing) when
 * the limit ran out; used to test failure detection without hanging a GPU. Synchronous. */
tg_status tg_bounded_wait_test(tg_ctx* ctx, const uint32_t* flag, int64_t limit_ns, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TG_H_ */
