// C ABI of the genome-scan library: argument checks, device memory of contexts and panels,
// tensor maps, stage timing and the orchestration of the kernels of one block scan.
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>

#include "internal.h"
#include "pvalue.cuh"

using namespace tg;

namespace {

thread_local std::string g_err;

const char* kVersion = "tg 0.1.0 (sm_103a)";

// The spin limit of device-side waits: generous enough for a FULL-output tile epilogue.
constexpr long long kSpinNs = 4000000000ll;
constexpr int kGroupDefault = 32;  // raster group (m-tiles) when the tuner has not chosen one

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

namespace tg {
// 2-D bf16 tensor map: rows x K elements, row stride ld elements, box box_rows x 32, 64B swizzle.
bool make_tmap(CUtensorMap* m, const void* ptr, int64_t rows, int64_t K, int64_t ld,
               uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {32u, box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
bool make_tmap_packed(CUtensorMap* m, const void* ptr, int64_t rows, int64_t ld, uint32_t box_bytes,
                      uint32_t box_rows, bool swizzle64) {
  if (swizzle64 && box_bytes != 64) return false;
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {box_bytes, box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
}  // namespace tg

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

#define TG_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

#define TG_ARG(cond, msg)                                   \
  do {                                                      \
    if (!(cond)) return fail(TG_ERR_INVALID_ARG, msg);      \
  } while (0)

// ---------------------------------------------------------------- profiling
// Each stage is also an NVTX range on the calling thread (named for profilers and timelines;
// a no-op when no tool is attached).
const char* const kStageNames[TG_N_STAGES] = {"tg.decode", "tg.project", "tg.norm",
                                              "tg.scan",   "tg.h2d",     "tg.stats"};
struct StageScope {
  tg_ctx* c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  StageScope(tg_ctx* c_, int s_, cudaStream_t st_, int nlaunch) : c(c_), stage(s_), st(st_) {
    nvtxRangePushA(kStageNames[stage]);
    c->launches[stage] += nlaunch;
    if (!c->prof) return;
    a = take();
    b = take();
    cudaEventRecord(a, st);
  }
  ~StageScope() {
    nvtxRangePop();
    if (!c->prof || !a) return;
    cudaEventRecord(b, st);
    c->pending.push_back({a, b, stage});
  }
  cudaEvent_t take() {
    if (!c->event_pool.empty()) {
      cudaEvent_t e = c->event_pool.back();
      c->event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

cudaError_t ensure_markers(tg_ctx* c, int64_t M) {
  if (M <= c->cap_m) return cudaSuccess;
  const int64_t cap = round_up(M, MT);
  dfree(c->nobs); dfree(c->mean); dfree(c->shift); dfree(c->mh); dfree(c->gc2s); dfree(c->gc2); dfree(c->qg);
  dfree(c->gres2); dfree(c->rinv); dfree(c->rinv64); dfree(c->refine_list);
  c->cap_m = 0;
  cudaError_t e;
  if ((e = dalloc(&c->nobs, cap)) || (e = dalloc(&c->mean, cap)) || (e = dalloc(&c->shift, cap)) ||
      (e = dalloc(&c->mh, cap)) || (e = dalloc(&c->gc2s, cap)) ||
      (e = dalloc(&c->gc2, cap)) || (e = dalloc(&c->qg, cap * JCOLS)) ||
      (e = dalloc(&c->gres2, cap)) || (e = dalloc(&c->rinv, cap)) || (e = dalloc(&c->rinv64, cap)) ||
      (e = dalloc(&c->refine_list, cap)))
    return e;
  c->cap_m = cap;
  return cudaSuccess;
}

// Operand rows: centred bf16 for the split form, float for FP32.
cudaError_t ensure_operands(tg_ctx* c, int64_t M, int64_t Npad, int prec) {
  const int64_t rows = round_up(M, MT);
  const bool fits = rows <= c->cap_rows && Npad <= c->cap_npad;
  const bool have = prec == TG_PREC_FP32 ? c->A32 != nullptr : c->Ahi != nullptr;
  if (fits && have) return cudaSuccess;
  const int64_t R = fits ? c->cap_rows : std::max(rows, c->cap_rows);
  const int64_t K = fits ? c->cap_npad : std::max(Npad, c->cap_npad);
  if (!fits) {
    dfree(c->Ahi); dfree(c->A32);
  }
  cudaError_t e = cudaSuccess;
  if (prec == TG_PREC_FP32 && !c->A32) e = dalloc(&c->A32, (size_t)(R * K));
  if (!e && prec == TG_PREC_SPLIT_BF16 && !c->Ahi) e = dalloc(&c->Ahi, (size_t)(R * K));
  if (e) return e;
  c->cap_rows = R;
  c->cap_npad = K;
  return cudaSuccess;
}

// Split-K of the one-CTA kernel for a block of M markers: for a panel of at most 64 phenotypes
// (64-column tiles) it is chosen by rule, for wider panels it is the tuned value. A split pays
// only while the tiles are fewer than the SMs; every split keeps at least one 1,024-sample chunk.
struct SplitChoice {
  int ks = 1;
  int64_t tiles = 0;
};
SplitChoice pick_split(const tg_ctx* c, const tg_panel* p, int64_t M, bool single,
                       bool projection = false) {
  SplitChoice r;
  const int64_t n_mt = (M + MT - 1) / MT;
  const bool narrow = projection || p->P <= 64;  // the projection has one 64-column tile
  r.tiles = n_mt * (narrow ? 1 : (p->P + 255) / 256);
  int ks = 1;
  if (narrow) {
    while (ks < 4 && r.tiles * ks * 2 <= c->sm_count) ks *= 2;
  } else if (single) {
    const int t = c->tune_split[tune_bucket(M)];
    ks = t > 1 ? t : 1;
  }
  const int chunks = (int)((p->Npad / 32 + kAccumChunkKB - 1) / kAccumChunkKB);
  while (ks > 1 && (ks > chunks || ks > c->sm_count)) ks /= 2;
  r.ks = ks;
  return r;
}
size_t split_bytes(const SplitChoice& sc) {
  return sc.ks > 1 ? (size_t)sc.tiles * (size_t)(sc.ks - 1) * (size_t)(MT * 256) * sizeof(float) : 0;
}
cudaError_t ensure_split(tg_ctx* c, const SplitChoice& sc) {
  const size_t need = split_bytes(sc);
  if (need > c->sk_ws_bytes) {
    dfree(c->sk_ws);
    c->sk_ws_bytes = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->sk_ws), need);
    if (e != cudaSuccess) return e;
    c->sk_ws_bytes = need;
  }
  if (sc.ks > 1 && sc.tiles > c->sk_cnt_cap) {
    dfree(c->sk_cnt);
    c->sk_cnt_cap = 0;
    cudaError_t e = dalloc(&c->sk_cnt, (size_t)sc.tiles);
    if (e != cudaSuccess) return e;
    c->sk_cnt_cap = sc.tiles;
  }
  return cudaSuccess;
}
bool split_fits(const tg_ctx* c, const SplitChoice& sc) {
  return split_bytes(sc) <= c->sk_ws_bytes && (sc.ks <= 1 || sc.tiles <= c->sk_cnt_cap);
}

// Size the context's workspace for the scans a graph will capture: nothing may allocate inside
// a capture. A workspace that another live graph has captured cannot move, so while one exists
// only a graph whose blocks fit the current buffers is accepted.
tg_status reserve_graph_workspace(tg_ctx* c, const tg_panel* p, int n_blocks, const int64_t* M,
                                  int64_t maxM, bool need_operand, const tg_scan_opts& opts) {
  const bool split = opts.precision == TG_PREC_SPLIT_BF16;
  std::vector<SplitChoice> need;
  for (int b = 0; b < n_blocks; ++b) {
    if (split && (p->P <= 64 || c->tune_kernel[tune_bucket(M[b])] == TUNE_SINGLE))
      need.push_back(pick_split(c, p, M[b], true));
    if (split && opts.mode == TG_MODE_PROJECTED && p->q > 1)
      need.push_back(pick_split(c, p, M[b], true, true));
  }
  if (c->graphs_alive > 0) {
    bool fits = maxM <= c->cap_m;
    if (need_operand)
      fits = fits && round_up(maxM, MT) <= c->cap_rows && p->Npad <= c->cap_npad &&
             (opts.precision == TG_PREC_FP32 ? c->A32 != nullptr : c->Ahi != nullptr);
    for (const SplitChoice& sc : need) fits = fits && split_fits(c, sc);
    if (!fits)
      return fail(TG_ERR_INVALID_ARG,
                  "another captured scan graph holds this context's workspace: capture the "
                  "largest blocks first, or use another context");
    return TG_OK;
  }
  TG_CUDA(ensure_markers(c, maxM));
  if (need_operand) TG_CUDA(ensure_operands(c, maxM, p->Npad, opts.precision));
  for (const SplitChoice& sc : need) TG_CUDA(ensure_split(c, sc));
  return TG_OK;
}

}  // namespace

namespace tg {

tg_status check_scan_args(const tg_ctx* c, const tg_panel* p, const ScanArgs& a) {
  TG_ARG(c && p, "null context or panel");
  TG_ARG(a.encoding == TG_ENC_2BIT || a.encoding == TG_ENC_U8_DOSAGE, "unknown encoding");
  TG_ARG(a.opts.precision == TG_PREC_FP32 || a.opts.precision == TG_PREC_SPLIT_BF16 ||
             a.opts.precision == TG_PREC_FP4_PIECES,
         "unknown precision");
  if (a.opts.precision == TG_PREC_FP4_PIECES) {
    if (a.encoding != TG_ENC_2BIT)
      return fail(TG_ERR_UNSUPPORTED, "the FP4 form scans 2-bit calls only (dosage bytes are not E2M1 values)");
    if (p->samples) return fail(TG_ERR_UNSUPPORTED, "the FP4 form does not scan subset panels");
  }
  TG_ARG(a.opts.mode == TG_MODE_PROJECTED || a.opts.mode == TG_MODE_PAPER, "unknown mode");
  TG_ARG(a.opts.reserved == 0, "tg_scan_opts.reserved must be 0");
  TG_ARG(a.opts.mode == TG_MODE_PROJECTED || a.N > 2, "the paper's form needs N > 2");
  TG_ARG(a.N == p->N, "N differs from the panel's sample count");
  TG_ARG(a.M >= 0, "M < 0");
  TG_ARG(a.marker_offset >= 0 && a.marker_offset + a.M <= 0xFFFFFFFFll,
         "marker indices must fit in 32 bits");
  if (a.M == 0) return TG_OK;
  TG_ARG(a.G != nullptr && aligned(a.G, 16), "G must be a 16-byte aligned device pointer");
  const int64_t need = a.encoding == TG_ENC_2BIT ? (a.N + 3) / 4 : a.N;
  TG_ARG(a.ldg >= need && a.ldg % 16 == 0, "ldg must be >= the packed row length and a multiple of 16");
  if (a.encoding == TG_ENC_2BIT)
    TG_ARG(a.missing == nullptr, "2-bit calls carry missingness in-band: missing must be NULL");
  if (a.missing) TG_ARG(a.ldm >= (a.N + 31) / 32 && aligned(a.missing, 4), "bad missing mask stride");
  if (a.opts.full_output) {
    TG_ARG(a.out.ldo >= p->P, "ldo < P");
    TG_ARG(a.out.beta || a.out.se || a.out.t || a.out.mlog10p, "full_output without output arrays");
  }
  const bool hits = a.opts.hit_mlog10p > 0.0;
  if (hits) TG_ARG(a.out.n_hits && a.out.hit_capacity >= 0 && (a.out.hits || a.out.hit_capacity == 0),
                   "hit collection needs hits, hit_capacity and n_hits");
  return TG_OK;
}

}  // namespace tg

namespace {

float r2_threshold(double mlog10p, double df, double lnB) {
  if (!(mlog10p > 0.0)) return 2.0f;  // never reached
  return (float)host_r2_threshold(mlog10p, df, lnB);
}

}  // namespace

namespace tg {

// The E2M1 pieces of a panel for the FP4 form, built on its first FP4 scan (synchronous).
tg_status ensure_fp4_panel(tg_ctx* c, tg_panel* p, cudaStream_t st) {
  if (p->fp4B) return TG_OK;
  if (c->graphs_alive > 0)
    return fail(TG_ERR_INVALID_ARG, "the FP4 pieces of a panel are built outside captured graphs");
  const int64_t Np = p->Npad, Pp = p->Ppad, nb = p->Npad / 2;
  cudaError_t e;
  auto undo = [&]() {
    dfree(p->fp4B); dfree(p->fp4B_scale); dfree(p->fp4B_cs);
    dfree(p->fp4Q); dfree(p->fp4Q_scale); dfree(p->fp4Q_cs);
    p->fp4B = nullptr; p->fp4Q = nullptr;
  };
  if ((e = dalloc(&p->fp4B, (size_t)(kFp4Pieces * Pp * nb))) || (e = dalloc(&p->fp4B_scale, (size_t)Pp)) ||
      (e = dalloc(&p->fp4B_cs, (size_t)Pp)) || (e = dalloc(&p->fp4Q, (size_t)(kFp4Pieces * QCOLS * nb))) ||
      (e = dalloc(&p->fp4Q_scale, (size_t)QCOLS)) || (e = dalloc(&p->fp4Q_cs, (size_t)QCOLS))) {
    undo();
    return cuda_fail(e, "FP4 panel pieces allocation");
  }
  if ((e = launch_fp4_pieces(p->Yres, p->N, p->s, p->col_rmul, p->P, Pp, p->N, Np, p->fp4B,
                             p->fp4B_scale, p->fp4B_cs, st)) ||
      (e = launch_fp4_pieces(p->Q + p->N, p->N, nullptr, nullptr, p->q - 1, QCOLS, p->N, Np, p->fp4Q,
                             p->fp4Q_scale, p->fp4Q_cs, st)) ||
      (e = cudaStreamSynchronize(st))) {
    undo();
    return cuda_fail(e, "FP4 panel pieces");
  }
  if (!make_tmap_packed(&p->tmFB, p->fp4B, kFp4Pieces * Pp, nb, 64u, 128u, true) ||
      !make_tmap_packed(&p->tmFQ, p->fp4Q, kFp4Pieces * QCOLS, nb, 64u, 64u, true)) {
    undo();
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the FP4 pieces");
  }
  return TG_OK;
}

// The FP4 form of a block scan (2-bit calls): a one-pass decode (the E2M1 operand and the row
// statistics), projection and contraction on kind::mxf4 tensor cores, norms (markers with a
// missing call untestable), then the same statistics as the split form.
tg_status scan_fp4(tg_ctx* c, tg_panel* p, const ScanArgs& a, cudaStream_t st) {
  const tg_status ps = ensure_fp4_panel(c, p, st);
  if (ps != TG_OK) return ps;
  TG_CUDA(ensure_markers(c, a.M));
  const int64_t lda = p->Npad / 2;
  const int64_t need = round_up(a.M, MT) * lda;
  if (need > c->cap_fp4) {
    if (c->graphs_alive > 0)
      return fail(TG_ERR_INVALID_ARG, "the context's workspace is held by a captured scan graph");
    dfree(c->Afp4);
    c->Afp4 = nullptr;
    c->cap_fp4 = 0;
    TG_CUDA(dalloc(&c->Afp4, (size_t)need));
    c->cap_fp4 = need;
  }
  {
    StageScope s(c, STAGE_DECODE, st, 1);
    TG_CUDA(launch_fp4_decode(a.G, a.ldg, a.N, a.M, c->Afp4, lda, c->nobs, c->mean, c->gc2,
                              c->shift, st));
  }
  CUtensorMap tA;
  if (!make_tmap_packed(&tA, c->Afp4, a.M, lda, 64u, (uint32_t)MT, true))
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the E2M1 operand");
  const int64_t nq = a.opts.mode == TG_MODE_PAPER ? 0 : p->q - 1;
  if (nq > 0) {
    StageScope s(c, STAGE_PROJECT, st, 1);
    EpiParams pp{};
    pp.M = (int)a.M;
    pp.P = (int)nq;
    pp.status = c->status;
    pp.row_shift = c->shift;
    pp.col_cs = p->fp4Q_cs;
    pp.col_rmul = p->fp4Q_scale;
    pp.raw_out = c->qg;
    pp.raw_cols = (int)nq;
    pp.raw_ld = QCOLS;
    TG_CUDA(launch_fp4_scan(&tA, &p->tmFQ, QCOLS, p->Npad, pp, c->sm_count, kSpinNs, st));
  }
  {
    StageScope s(c, STAGE_NORM, st, nq > 0 ? 2 : 1);
    const MarkerRefine rf{a.G, a.ldg, a.encoding, a.N, nullptr, 0, c->mean, p->Q, (int)p->q,
                          c->refine_list, c->scratch + 40};
    TG_CUDA(launch_marker_norm(a.M, c->nobs, c->gc2, c->qg, QCOLS, nq, 1.0, c->gres2,
                               a.out.marker_norm2, c->rinv, c->rinv64, &rf, st, a.N));
    if (a.out.marker_nobs)
      TG_CUDA(cudaMemcpyAsync(a.out.marker_nobs, c->nobs, sizeof(int32_t) * a.M,
                              cudaMemcpyDeviceToDevice, st));
    if (a.out.marker_mean)
      TG_CUDA(cudaMemcpyAsync(a.out.marker_mean, c->mean, sizeof(double) * a.M,
                              cudaMemcpyDeviceToDevice, st));
  }
  EpiParams ep{};
  ep.M = (int)a.M;
  ep.P = (int)p->P;
  ep.marker_offset = a.marker_offset;
  mode_df(p, a.opts.mode, &ep.df, &ep.lnB);
  ep.df_f = (float)ep.df;
  ep.kappa = 1.0f;
  ep.kappa64 = 1.0;
  ep.do_hits = a.opts.hit_mlog10p > 0.0 && a.out.n_hits != nullptr;
  ep.r2_thr = ep.do_hits ? (float)host_r2_threshold(a.opts.hit_mlog10p, ep.df, ep.lnB) : 2.0f;
  ep.do_full = a.opts.full_output ? 1 : 0;
  ep.do_best = a.out.best != nullptr;
  ep.row_inv = c->rinv;
  ep.row_inv64 = c->rinv64;
  ep.exact = ExactArgs{a.G, a.ldg, a.encoding, (int)a.N, nullptr, 0, c->mean, p->Yres, p->N};
  ep.col_s = p->col_s;
  ep.col_s64 = p->s;
  ep.col_rmul = p->fp4B_scale;  // 2^-e of each column's pieces, NaN for an untestable phenotype
  ep.row_shift = c->shift;      // -mean: the centring add-back
  ep.col_cs = p->fp4B_cs;
  ep.beta = a.out.beta;
  ep.se = a.out.se;
  ep.t = a.out.t;
  ep.mlp = a.out.mlog10p;
  ep.rstore = a.out.t ? a.out.t : a.out.mlog10p ? a.out.mlog10p : a.out.beta ? a.out.beta : a.out.se;
  ep.ldo = a.out.ldo;
  ep.hits = a.out.hits;
  ep.hit_cap = a.out.hit_capacity;
  ep.n_hits = a.out.n_hits;
  ep.best = a.out.best;
  ep.status = c->status;
  unsigned long long* hit_start = reinterpret_cast<unsigned long long*>(c->scratch + 16);
  if (ep.do_hits)
    TG_CUDA(cudaMemcpyAsync(hit_start, ep.n_hits, sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, st));
  {
    StageScope s(c, STAGE_GEMM, st, 1);
    TG_CUDA(launch_fp4_scan(&tA, &p->tmFB, (int)p->Ppad, p->Npad, ep, c->sm_count, kSpinNs, st));
  }
  if (ep.do_hits || ep.do_full) {
    StageScope s(c, STAGE_STATS, st, (ep.do_hits ? 1 : 0) + (ep.do_full ? 1 : 0));
    if (ep.do_hits) TG_CUDA(launch_hit_stats(ep, hit_start, st));
    if (ep.do_full) TG_CUDA(launch_full_stats(ep, st));
  }
  return TG_OK;
}

tg_status scan_impl(tg_ctx* c, const tg_panel* pc, const ScanArgs& a, cudaStream_t st) {
  tg_panel* p = const_cast<tg_panel*>(pc);
  if (a.M == 0) return TG_OK;
  if (a.opts.precision == TG_PREC_FP4_PIECES) return scan_fp4(c, p, a, st);
  const int prec = a.opts.precision;
  const bool split = prec == TG_PREC_SPLIT_BF16;
  // a small panel's joint projection pass (projected form, joint operand of at most 128 rows,
  // at least one 128-marker tile per SM) reads the packed rows and decodes them in shared memory
  const bool fuse_joint = split && c->fuse_joint && a.missing == nullptr &&
                          a.opts.mode == TG_MODE_PROJECTED && p->q > 1 && p->joint_cols > 0 &&
                          p->joint_cols <= 128 && p->QYhi16 != nullptr &&
                          (a.M + MT - 1) / MT >= c->sm_count;
  // a larger panel's projection (P + q - 1 > 128, same conditions otherwise): the same pass with
  // the 64 projection columns alone reads the packed rows and also writes the block's operand
  // as it expands them, so the operand is written once and read once (by the panel's
  // contraction) instead of being read a second time for the projection. A panel with a
  // 256-row joint operand keeps its one joint pass over the decoded operand unless this pass
  // also takes the statistics (dosage rows on 256-marker tiles): with a counting pass first the
  // projection and the contraction as two passes take longer than the decode and one pass.
  const bool one_pass_rows = a.encoding == TG_ENC_U8_DOSAGE && a.N <= kOnePassMaxN &&
                             joint_fused_rows(a.M, c->sm_count, QCOLS) == 2 * MT;
  const bool fuse_proj = split && c->fuse_joint && !c->fuse_decode && !fuse_joint &&
                         a.missing == nullptr && a.opts.mode == TG_MODE_PROJECTED && p->q > 1 &&
                         p->QBhi16 != nullptr && (a.M + MT - 1) / MT >= c->sm_count &&
                         (p->joint_cols == 0 || one_pass_rows);
  // split-form 2-bit blocks and unmasked dosage blocks are decoded inside the contraction
  // kernels when the context asks for it; the rest go through a decoded operand in HBM
  const bool fused = split && a.missing == nullptr && (c->fuse_decode || fuse_joint);
  if (c->graphs_alive > 0) {
    const bool grow = a.M > c->cap_m || (!fused && (round_up(a.M, MT) > c->cap_rows ||
                                                    p->Npad > c->cap_npad ||
                                                    (prec == TG_PREC_FP32 ? !c->A32 : !c->Ahi)));
    const int bq = tune_bucket(a.M);
    const bool single = split && (p->P <= 64 || c->tune_kernel[bq] == TUNE_SINGLE);
    const bool proj = split && a.opts.mode == TG_MODE_PROJECTED && p->q > 1;
    if (grow || (single && !split_fits(c, pick_split(c, p, a.M, true))) ||
        (proj && !split_fits(c, pick_split(c, p, a.M, true, true))))
      return fail(TG_ERR_INVALID_ARG,
                  "the context's workspace is held by a captured scan graph: scan blocks no "
                  "larger than the graph's, or use another context");
  }
  TG_CUDA(ensure_markers(c, a.M));
  if (!fused) TG_CUDA(ensure_operands(c, a.M, p->Npad, prec));
  const double kappa64 = a.encoding == TG_ENC_U8_DOSAGE ? 2.0 / 255.0 : 1.0;
  const float kappa = (float)kappa64;
  void* Ahi = fused ? nullptr : prec == TG_PREC_FP32 ? (void*)c->A32 : (void*)c->Ahi;
  // dosage rows in the joint pass (or the projection pass that writes the operand) on 256-row
  // tiles: that pass writes the row statistics itself (a thread holds a whole row), so no
  // counting pass reads the block first
  const int pass_cols = fuse_proj ? QCOLS : p->joint_cols;
  const bool one_pass = (fuse_joint || fuse_proj) && a.encoding == TG_ENC_U8_DOSAGE &&
                        a.N <= kOnePassMaxN &&
                        joint_fused_rows(a.M, c->sm_count, pass_cols) == 2 * MT;
  if (!one_pass) {  // (a counting pass alone before the projection pass that writes the operand)
    StageScope s(c, STAGE_DECODE, st, 1);
    TG_CUDA(launch_decode(a.G, a.ldg, a.encoding, a.N, a.M, a.missing, a.ldm, prec,
                          fuse_proj ? nullptr : Ahi, split ? c->shift : nullptr,
                          split ? c->mh : nullptr, p->Npad, c->nobs, nullptr, nullptr, c->mean,
                          c->gc2, st));
  }
  DecodeArgs da{}, dj{};
  if (fused || fuse_proj) {
    da.N = (int)a.N;
    da.M = (int)a.M;
    da.shift = c->shift;
    da.mh = c->mh;
    dj = da;
    if (one_pass) {
      dj.shift_out = c->shift;
      dj.nobs_out = c->nobs;
      dj.mean_out = c->mean;
      dj.gc2_out = c->gc2;
    }
    if (fuse_proj) {
      dj.a_out = c->Ahi;
      dj.lda_out = p->Npad;
    }
    const bool u8 = a.encoding == TG_ENC_U8_DOSAGE;
    if ((fused && !make_tmap_packed(&da.tmG, a.G, a.M, a.ldg, u8 ? 32u : 16u)) ||
        ((fuse_joint || fuse_proj) &&
         !make_tmap_packed(&dj.tmG, a.G, a.M, a.ldg, u8 ? 64u : 16u,
                           (uint32_t)joint_fused_rows(a.M, c->sm_count, pass_cols), u8)))
      return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the packed genotypes");
  }
  const DecodeArgs* dec = fused ? &da : nullptr;
  const int64_t nq = a.opts.mode == TG_MODE_PAPER ? 0 : p->q - 1;
  CUtensorMap tA;
  if (split && !fused && !make_tmap(&tA, c->Ahi, a.M, p->Npad, p->Npad, MT))
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the genotype operand");
  // a small panel in the projected form: one pass over the operand gives the projection and the
  // panel's products (raw, into qg after the projection columns); the statistics follow the norms
  const bool joint = split && nq > 0 && p->joint_cols > 0 && !fuse_proj;
  const int64_t ldq = joint ? p->joint_cols : QCOLS;  // qg row stride
  if (nq > 0) {
    StageScope s(c, STAGE_PROJECT, st, 1);
    if (!split) {
      TG_CUDA(launch_project(c->A32, p->Npad, a.M, p->Npad, p->QB, nq, c->qg, st));
    } else {
      EpiParams pp{};
      pp.M = (int)a.M;
      pp.P = (int)(joint ? nq + p->P : nq);
      pp.status = c->status;
      pp.row_shift = c->shift;
      pp.col_cs = joint ? p->qycs : p->qcs;
      pp.raw_out = c->qg;
      pp.raw_cols = pp.P;
      pp.raw_ld = (int)ldq;
      if (fuse_joint) {
        const bool u8 = a.encoding == TG_ENC_U8_DOSAGE;  // dosage rows: the f16 joint operand
        if (u8) pp.col_cs = p->qycs16;
        TG_CUDA(launch_joint_fused(u8 ? &p->tmQYhi16 : &p->tmQYhi, u8 ? &p->tmQYlo16 : &p->tmQYlo,
                                   p->Npad, pp, c->sm_count, kSpinNs, st, dj, a.encoding));
      } else if (fuse_proj) {  // the projection alone, writing the operand as it goes
        const bool u8 = a.encoding == TG_ENC_U8_DOSAGE;
        if (u8) pp.col_cs = p->qcs16;
        TG_CUDA(launch_joint_fused(u8 ? &p->tmQhi16 : &p->tmQhi, u8 ? &p->tmQlo16 : &p->tmQlo,
                                   p->Npad, pp, c->sm_count, kSpinNs, st, dj, a.encoding));
      } else {
        const SplitChoice sc = pick_split(c, p, a.M, true, true);
        if (sc.ks > 1) {  // a small block: split K so that more SMs stream the operand
          TG_CUDA(ensure_split(c, sc));
          pp.ksplit = sc.ks;
          pp.sk_ws = c->sk_ws;
          pp.sk_cnt = c->sk_cnt;
          TG_CUDA(cudaMemsetAsync(pp.sk_cnt, 0, sizeof(unsigned) * (size_t)sc.tiles, st));
        }
        TG_CUDA(launch_tc_scan(&tA, joint ? &p->tmQYhi : &p->tmQhi, joint ? &p->tmQYlo : &p->tmQlo,
                               p->Npad, pp, c->sm_count, kSpinNs, st, kGroupDefault,
                               c->fuse_decode ? dec : nullptr, a.encoding));
      }
    }
  }
  if (p->samples) {  // a subset panel: |g_c|^2 over its samples
    StageScope s(c, STAGE_NORM, st, 1);
    TG_CUDA(launch_subset_stats(a.G, a.ldg, a.encoding, a.N, a.M, a.missing, a.ldm, p->samples,
                                c->mean, c->gc2s, st));
  }
  {
    StageScope s(c, STAGE_NORM, st, nq > 0 ? 2 : 1);
    const MarkerRefine rf{a.G, a.ldg, a.encoding, a.N, a.missing, a.ldm, c->mean, p->Q, (int)p->q,
                          c->refine_list, c->scratch + 40};
    TG_CUDA(launch_marker_norm(a.M, c->nobs, p->samples ? c->gc2s : c->gc2, c->qg, ldq, nq, kappa64, c->gres2,
                               a.out.marker_norm2, c->rinv, c->rinv64, &rf, st));
    if (a.out.marker_nobs)
      TG_CUDA(cudaMemcpyAsync(a.out.marker_nobs, c->nobs, sizeof(int32_t) * a.M,
                              cudaMemcpyDeviceToDevice, st));
    if (a.out.marker_mean)
      TG_CUDA(cudaMemcpyAsync(a.out.marker_mean, c->mean, sizeof(double) * a.M,
                              cudaMemcpyDeviceToDevice, st));
  }
  EpiParams ep{};
  ep.M = (int)a.M;
  ep.P = (int)p->P;
  ep.marker_offset = a.marker_offset;
  mode_df(p, a.opts.mode, &ep.df, &ep.lnB);
  ep.df_f = (float)ep.df;
  ep.kappa = kappa;
  ep.kappa64 = kappa64;
  ep.do_hits = a.opts.hit_mlog10p > 0.0 && a.out.n_hits != nullptr;
  ep.r2_thr = ep.do_hits ? r2_threshold(a.opts.hit_mlog10p, ep.df, ep.lnB) : 2.0f;
  ep.do_full = a.opts.full_output ? 1 : 0;
  ep.do_best = a.out.best != nullptr;
  ep.row_inv = c->rinv;
  ep.row_inv64 = c->rinv64;
  ep.exact = ExactArgs{a.G, a.ldg, a.encoding, (int)a.N, a.missing, a.ldm, c->mean, p->Yres, p->N};
  ep.col_s = p->col_s;
  ep.col_s64 = p->s;
  ep.col_rmul = p->col_rmul;
  ep.row_shift = split ? c->shift : nullptr;
  ep.col_cs = p->col_cs;
  ep.beta = a.out.beta;
  ep.se = a.out.se;
  ep.t = a.out.t;
  ep.mlp = a.out.mlog10p;
  ep.rstore = a.out.t ? a.out.t : a.out.mlog10p ? a.out.mlog10p : a.out.beta ? a.out.beta : a.out.se;
  ep.ldo = a.out.ldo;
  ep.hits = a.out.hits;
  ep.hit_cap = a.out.hit_capacity;
  ep.n_hits = a.out.n_hits;
  ep.best = a.out.best;
  ep.status = c->status;
  unsigned long long* hit_start = reinterpret_cast<unsigned long long*>(c->scratch + 16);
  if (ep.do_hits)
    TG_CUDA(cudaMemcpyAsync(hit_start, ep.n_hits, sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, st));
  {
    StageScope s(c, STAGE_GEMM, st, 1);
    if (prec == TG_PREC_FP32) {
      TG_CUDA(launch_sgemm_scan(c->A32, p->Npad, p->B32, p->Npad, p->Npad, ep, st));
    } else if (joint) {  // the products came with the projection
      TG_CUDA(launch_raw_stats(c->qg + nq, ldq, ep, st));
    } else {
      const int b = tune_bucket(a.M);
      const int group = c->tune_group[b] > 0 ? c->tune_group[b] : kGroupDefault;
      const bool narrow = p->P <= 64;  // a small panel: 64-column tiles, bound by HBM
      if (narrow || c->tune_kernel[b] == TUNE_SINGLE) {
        const SplitChoice sc = pick_split(c, p, a.M, true);
        if (sc.ks > 1) {  // split-K while the tiles are fewer than the SMs
          TG_CUDA(ensure_split(c, sc));
          ep.ksplit = sc.ks;
          ep.sk_ws = c->sk_ws;
          ep.sk_cnt = c->sk_cnt;
          TG_CUDA(cudaMemsetAsync(ep.sk_cnt, 0, sizeof(unsigned) * (size_t)sc.tiles, st));
        }
        TG_CUDA(launch_tc_scan(&tA, narrow ? &p->tmBhi64 : &p->tmBhi, narrow ? &p->tmBlo64 : &p->tmBlo,
                               p->Npad, ep, c->sm_count, kSpinNs, st, group, dec, a.encoding, narrow));
      }
      else {
        ep.wave_ctr = reinterpret_cast<unsigned long long*>(c->scratch + 32);
        TG_CUDA(cudaMemsetAsync(ep.wave_ctr, 0, sizeof(unsigned long long), st));
        TG_CUDA(launch_tc2_scan(&tA, &p->tmBhi2, &p->tmBlo2, p->Npad, ep, c->sm_count, kSpinNs, st,
                                group, dec, a.encoding));
      }
    }
  }
  if (ep.do_hits || ep.do_full) {
    StageScope s(c, STAGE_STATS, st, (ep.do_hits ? 1 : 0) + (ep.do_full ? 1 : 0));
    if (ep.do_hits) TG_CUDA(launch_hit_stats(ep, hit_start, st));
    if (ep.do_full) TG_CUDA(launch_full_stats(ep, st));
  }
  return TG_OK;
}

}  // namespace tg

namespace tg {

void mode_df(const tg_panel* p, int mode, double* df, double* lnB) {
  if (mode == TG_MODE_PAPER) {
    *df = (double)(p->NS - 2);
    *lnB = p->lnB_paper;
  } else {
    *df = (double)p->df;
    *lnB = p->lnB;
  }
}

tg_status fail(tg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

tg_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA;
}

double host_lnbeta_half(double df) {
  const double a = 0.5 * df;
  return std::lgamma(a) + std::lgamma(0.5) - std::lgamma(a + 0.5);
}

// Smallest r^2 whose -log10 p reaches the threshold (bisection on |r|, monotone in |r|).
double host_r2_threshold(double mlog10p, double df, double lnB) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (mlog10p_r(mid, df, lnB) >= mlog10p) hi = mid; else lo = mid;
  }
  return hi * hi;
}

}  // namespace tg

struct tg_graph {
  tg_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches[TG_N_STAGES] = {0, 0, 0, 0, 0, 0};
  uint8_t* stage[2] = {nullptr, nullptr};  // device staging of host blocks (host-block graphs)
};

extern "C" {

const char* tg_version(void) { return kVersion; }
int tg_abi_version(void) { return TG_ABI_VERSION; }
const char* tg_last_error(void) { return g_err.c_str(); }

const char* tg_status_string(tg_status s) {
  switch (s) {
    case TG_OK: return "ok";
    case TG_ERR_INVALID_ARG: return "invalid argument";
    case TG_ERR_CUDA: return "CUDA error";
    case TG_ERR_OOM: return "out of device memory";
    case TG_ERR_NONFINITE: return "non-finite input";
    case TG_ERR_RANK: return "too few samples for the covariate rank";
    case TG_ERR_CAPACITY: return "hit buffer overflow";
    case TG_ERR_TIMEOUT: return "device wait timed out";
    case TG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

tg_status tg_create(tg_ctx** out, int device) {
  TG_ARG(out != nullptr, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  TG_CUDA(cudaGetDeviceCount(&ndev));
  TG_ARG(device >= 0 && device < ndev, "no such CUDA device");
  TG_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  TG_CUDA(cudaGetDeviceProperties(&prop, device));
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(TG_ERR_UNSUPPORTED, std::string("needs an sm_103 (GB300) device, found ") + prop.name);
  if (!encode_fn()) return fail(TG_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  tg_ctx* c = new tg_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) ||
      (e = dalloc(&c->status, 4)) || (e = dalloc(&c->scratch, 256)) ||
      (e = cudaMemset(c->status, 0, 16))) {
    tg_destroy(c);
    return cuda_fail(e, "tg_create");
  }
  for (int i = 0; i < 4 * kRateBlocks; ++i)
    if ((e = cudaEventCreate(&c->ev_rate[i]))) {
      tg_destroy(c);
      return cuda_fail(e, "tg_create");
    }
  if ((e = cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming))) {
    tg_destroy(c);
    return cuda_fail(e, "tg_create");
  }
  for (int i = 0; i < kRingEvents; ++i)
    if ((e = cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming))) {
      tg_destroy(c);
      return cuda_fail(e, "tg_create");
    }
  *out = c;
  return TG_OK;
}

tg_status tg_destroy(tg_ctx* c) {
  if (!c) return TG_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  dfree(c->status); dfree(c->scratch);
  dfree(c->Ahi); dfree(c->A32); dfree(c->Afp4); dfree(c->shift); dfree(c->mh); dfree(c->gc2s);
  dfree(c->nobs); dfree(c->mean); dfree(c->gc2); dfree(c->qg); dfree(c->gres2);
  dfree(c->rinv); dfree(c->rinv64); dfree(c->refine_list);
  dfree(c->sk_ws); dfree(c->sk_cnt);
  dfree(c->stage);
  dfree(c->dhits); dfree(c->dnhits); dfree(c->dbest);
  for (auto& ev : c->pending) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
  for (auto ev : c->event_pool) cudaEventDestroy(ev);
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);
  for (int i = 0; i < kRingEvents; ++i)
    if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
  for (int i = 0; i < 4 * kRateBlocks; ++i)
    if (c->ev_rate[i]) cudaEventDestroy(c->ev_rate[i]);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
  return TG_OK;
}

// The joint operand of a small panel (tg_panel::QYhi): the q - 1 projection rows, then the P
// phenotype rows, copied from the panel's own split operands, in the fewest of 64, 128 or 256
// rows that hold them. Nothing for a panel without covariate columns or with P + q - 1 > 256.
// A panel with P + q - 1 > 128 gets the f16 copy of its projection columns alone instead of the
// joint f16 operand (tg_panel::QBhi16). Synchronous on st.
tg_status build_joint(tg_panel* p, cudaStream_t st) {
  const int64_t nq = p->q - 1, P = p->P, Np = p->Npad;
  if (nq <= 0 || P <= 0) return TG_OK;
  cudaError_t e;
  if (P + nq > 128) {  // the projection pass that also writes the operand reads these
    if ((e = dalloc(&p->QBhi16, (size_t)(QCOLS * Np))) ||
        (e = dalloc(&p->QBlo16, (size_t)(QCOLS * Np))) || (e = dalloc(&p->qcs16, (size_t)QCOLS)) ||
        (e = launch_joint_f16(p->Q, p->N, nq, p->Yres, p->s, p->col_rmul, 0, QCOLS, Np, p->QBhi16,
                              p->QBlo16, p->qcs16, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "f16 projection operand");
    if (!make_tmap(&p->tmQhi16, p->QBhi16, QCOLS, Np, Np, QCOLS) ||
        !make_tmap(&p->tmQlo16, p->QBlo16, QCOLS, Np, Np, QCOLS))
      return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the f16 projection operand");
  }
  if (P + nq > JCOLS) return TG_OK;
  const int64_t jc = P + nq <= 64 ? 64 : P + nq <= 128 ? 128 : 256;
  const size_t row = sizeof(__nv_bfloat16) * (size_t)Np;
  const auto d2d = cudaMemcpyDeviceToDevice;
  if ((e = dalloc(&p->QYhi, (size_t)(jc * Np))) || (e = dalloc(&p->QYlo, (size_t)(jc * Np))) ||
      (e = dalloc(&p->qycs, (size_t)jc)) ||
      (e = cudaMemsetAsync(p->QYhi, 0, row * jc, st)) ||
      (e = cudaMemsetAsync(p->QYlo, 0, row * jc, st)) ||
      (e = cudaMemsetAsync(p->qycs, 0, sizeof(float) * jc, st)) ||
      (e = cudaMemcpyAsync(p->QYhi, p->QBhi, row * nq, d2d, st)) ||
      (e = cudaMemcpyAsync(p->QYlo, p->QBlo, row * nq, d2d, st)) ||
      (e = cudaMemcpyAsync(p->QYhi + nq * Np, p->Bhi, row * P, d2d, st)) ||
      (e = cudaMemcpyAsync(p->QYlo + nq * Np, p->Blo, row * P, d2d, st)) ||
      (e = cudaMemcpyAsync(p->qycs, p->qcs, sizeof(float) * nq, d2d, st)) ||
      (e = cudaMemcpyAsync(p->qycs + nq, p->col_cs, sizeof(float) * P, d2d, st)) ||
      (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, "joint projection and panel operand");
  if (!make_tmap(&p->tmQYhi, p->QYhi, jc, Np, Np, (uint32_t)jc) ||
      !make_tmap(&p->tmQYlo, p->QYlo, jc, Np, Np, (uint32_t)jc))
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the joint operand");
  if (jc <= 128) {  // the f16 copy for the joint pass that decodes dosage rows in shared memory
    if ((e = dalloc(&p->QYhi16, (size_t)(jc * Np))) || (e = dalloc(&p->QYlo16, (size_t)(jc * Np))) ||
        (e = dalloc(&p->qycs16, (size_t)jc)) ||
        (e = launch_joint_f16(p->Q, p->N, nq, p->Yres, p->s, p->col_rmul, P, jc, Np, p->QYhi16,
                              p->QYlo16, p->qycs16, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "f16 joint projection and panel operand");
    // 2-byte elements: the bf16 map layout serves (TMA copies bytes, it converts nothing)
    if (!make_tmap(&p->tmQYhi16, p->QYhi16, jc, Np, Np, (uint32_t)jc) ||
        !make_tmap(&p->tmQYlo16, p->QYlo16, jc, Np, Np, (uint32_t)jc))
      return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the f16 joint operand");
  }
  p->joint_cols = (int)jc;
  return TG_OK;
}

tg_status tg_prepare_panel(tg_ctx* c, const float* Y, int64_t ldy, int64_t N, int64_t P,
                           const double* C, int64_t ldc, int64_t n_cov, tg_panel** out,
                           void* stream) {
  TG_ARG(c && out, "null context or output");
  *out = nullptr;
  TG_ARG(N > 0 && P >= 0 && n_cov >= 0, "bad sizes");
  TG_ARG(N <= (1ll << 30), "N too large");
  TG_ARG(Y != nullptr || P == 0, "null Y");
  TG_ARG(ldy >= N, "ldy < N");
  if (n_cov > QMAX - 1) return fail(TG_ERR_UNSUPPORTED, "at most 63 covariates");
  if (n_cov > 0) TG_ARG(C != nullptr && ldc >= N, "null C or ldc < N");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  tg_panel* p = new tg_panel();
  p->device = c->device;
  p->N = N;
  p->P = P;
  p->n_cov = n_cov;
  p->NS = N;
  p->Npad = round_up(N, KPAD);
  p->Ppad = round_up(std::max<int64_t>(P, 1), PPAD);
  const int64_t k = 1 + n_cov;
  auto cleanup = [&](tg_status s) { tg_panel_free(p); return s; };
  cudaError_t e;
  int* dint = nullptr;  // [0] rank, [1..k] kept flags
  if ((e = dalloc(&p->X, (size_t)(2 * k * N))) || (e = dalloc(&p->Q, (size_t)(k * N))) ||
      (e = dalloc(&p->Yres, (size_t)(std::max<int64_t>(P, 1) * N))) ||
      (e = dalloc(&p->s, (size_t)std::max<int64_t>(P, 1))) ||
      (e = dalloc(&p->col_s, (size_t)std::max<int64_t>(P, 1))) ||
      (e = dalloc(&p->col_rmul, (size_t)p->Ppad)) || (e = dalloc(&p->col_cs, (size_t)p->Ppad)) ||
      (e = dalloc(&p->qcs, (size_t)QCOLS)) ||
      (e = dalloc(&p->Bhi, (size_t)(p->Ppad * p->Npad))) ||
      (e = dalloc(&p->Blo, (size_t)(p->Ppad * p->Npad))) ||
      (e = dalloc(&p->B32, (size_t)(p->Ppad * p->Npad))) ||
      (e = dalloc(&p->QB, (size_t)(QCOLS * p->Npad))) ||
      (e = dalloc(&p->QBhi, (size_t)(QCOLS * p->Npad))) ||
      (e = dalloc(&p->QBlo, (size_t)(QCOLS * p->Npad))) || (e = dalloc(&dint, (size_t)(1 + k))))
    return cleanup(cuda_fail(e, "tg_prepare_panel allocation"));
  auto run = [&]() -> cudaError_t {
    cudaError_t r;
    if ((r = cudaMemsetAsync(c->scratch, 0, 16, st))) return r;
    if ((r = cudaMemsetAsync(p->Bhi, 0, sizeof(__nv_bfloat16) * p->Ppad * p->Npad, st))) return r;
    if ((r = cudaMemsetAsync(p->Blo, 0, sizeof(__nv_bfloat16) * p->Ppad * p->Npad, st))) return r;
    if ((r = cudaMemsetAsync(p->B32, 0, sizeof(float) * p->Ppad * p->Npad, st))) return r;
    if ((r = cudaMemsetAsync(p->col_rmul, 0, sizeof(float) * p->Ppad, st))) return r;
    if ((r = cudaMemsetAsync(p->col_cs, 0, sizeof(float) * p->Ppad, st))) return r;
    if ((r = launch_build_design(p->X, C, ldc, N, n_cov, c->scratch, st))) return r;
    if ((r = launch_householder(p->X, N, k, p->Q, dint, dint + 1, st))) return r;
    return cudaSuccess;
  };
  if ((e = run())) { cudaFree(dint); return cleanup(cuda_fail(e, "tg_prepare_panel basis")); }
  int rank = 0;
  if ((e = cudaMemcpyAsync(&rank, dint, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st))) {
    cudaFree(dint);
    return cleanup(cuda_fail(e, "tg_prepare_panel rank"));
  }
  cudaFree(dint);
  p->q = rank;
  p->df = N - rank - 1;
  if (p->df <= 0) return cleanup(fail(TG_ERR_RANK, "N must exceed rank([1, C]) + 1"));
  if ((e = launch_residualise(Y, ldy, p->Q, N, P, rank, p->Npad, p->Yres, p->s, p->col_s,
                              p->col_rmul, p->Bhi, p->Blo, p->B32, p->col_cs, c->scratch, st)) ||
      (e = launch_qcols(p->Q, N, rank, p->Npad, p->QB, p->QBhi, p->QBlo, p->qcs, st)))
    return cleanup(cuda_fail(e, "tg_prepare_panel residualise"));
  uint32_t flags = 0;
  if ((e = cudaMemcpyAsync(&flags, c->scratch, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return cleanup(cuda_fail(e, "tg_prepare_panel"));
  if (flags & 1u) return cleanup(fail(TG_ERR_NONFINITE, "non-finite covariate"));
  if (flags & 2u) return cleanup(fail(TG_ERR_NONFINITE, "non-finite phenotype"));
  p->lnB = host_lnbeta_half((double)p->df);
  p->lnB_paper = host_lnbeta_half((double)(N - 2));
  if (!make_tmap(&p->tmBhi, p->Bhi, p->Ppad, p->Npad, p->Npad, 256) ||
      !make_tmap(&p->tmBlo, p->Blo, p->Ppad, p->Npad, p->Npad, 256) ||
      !make_tmap(&p->tmBhi2, p->Bhi, p->Ppad, p->Npad, p->Npad, 128) ||
      !make_tmap(&p->tmBlo2, p->Blo, p->Ppad, p->Npad, p->Npad, 128) ||
      !make_tmap(&p->tmQhi, p->QBhi, QCOLS, p->Npad, p->Npad, 64) ||
      !make_tmap(&p->tmQlo, p->QBlo, QCOLS, p->Npad, p->Npad, 64) ||
      !make_tmap(&p->tmBhi64, p->Bhi, p->Ppad, p->Npad, p->Npad, 64) ||
      !make_tmap(&p->tmBlo64, p->Blo, p->Ppad, p->Npad, p->Npad, 64))
    return cleanup(fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the panel"));
  const tg_status js = build_joint(p, st);
  if (js != TG_OK) return cleanup(js);
  *out = p;
  return TG_OK;
}

tg_status tg_prepare_panel_subset(tg_ctx* c, const float* Y, int64_t ldy, int64_t N, int64_t P,
                                  const double* C, int64_t ldc, int64_t n_cov,
                                  const uint32_t* samples, tg_panel** out, void* stream) {
  TG_ARG(c && out && samples, "null context, output or sample mask");
  *out = nullptr;
  TG_ARG(N > 0 && P >= 0 && n_cov >= 0, "bad sizes");
  TG_ARG(N <= (1ll << 30), "N too large");
  TG_ARG(Y != nullptr || P == 0, "null Y");
  TG_ARG(ldy >= N, "ldy < N");
  if (n_cov > 0) TG_ARG(C != nullptr && ldc >= N, "null C or ldc < N");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nw = (N + 31) / 32;
  std::vector<uint32_t> hm((size_t)nw);
  TG_CUDA(cudaMemcpyAsync(hm.data(), samples, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost, st));
  TG_CUDA(cudaStreamSynchronize(st));
  std::vector<int> idx;
  for (int64_t i = 0; i < N; ++i)
    if ((hm[(size_t)(i >> 5)] >> (i & 31)) & 1u) idx.push_back((int)i);
  const int64_t NS = (int64_t)idx.size();
  if (NS < 3) return fail(TG_ERR_RANK, "a subset panel needs at least 3 samples");
  int* didx = nullptr;
  float* Yc = nullptr;
  double* Cc = nullptr;
  tg_panel* pc = nullptr;
  tg_panel* r = nullptr;
  auto cleanup = [&](tg_status s) {
    dfree(didx); dfree(Yc); dfree(Cc);
    if (pc) tg_panel_free(pc);
    if (r) tg_panel_free(r);
    return s;
  };
  cudaError_t e;
  if ((e = dalloc(&didx, (size_t)NS)) || (e = dalloc(&Yc, (size_t)(std::max<int64_t>(P, 1) * NS))) ||
      (n_cov > 0 && (e = dalloc(&Cc, (size_t)(n_cov * NS)))))
    return cleanup(cuda_fail(e, "tg_prepare_panel_subset allocation"));
  if ((e = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * NS, cudaMemcpyHostToDevice, st)) ||
      (e = launch_gather_f32(Y, ldy, Yc, NS, didx, NS, P, st)) ||
      (n_cov > 0 && (e = launch_gather_f64(C, ldc, Cc, NS, didx, NS, n_cov, st))))
    return cleanup(cuda_fail(e, "tg_prepare_panel_subset gather"));
  // the panel on the gathered rows, then its sample-indexed arrays back on the full axis
  tg_status s = tg_prepare_panel(c, Yc, NS, NS, P, Cc, NS, n_cov, &pc, stream);
  if (s != TG_OK) return cleanup(s);
  r = new tg_panel();
  r->device = c->device;
  r->N = N;
  r->NS = NS;
  r->P = P;
  r->n_cov = n_cov;
  r->q = pc->q;
  r->df = pc->df;
  r->Npad = round_up(N, KPAD);
  r->Ppad = pc->Ppad;
  r->lnB = pc->lnB;
  r->lnB_paper = pc->lnB_paper;
  const int64_t Np = r->Npad, Pp = r->Ppad, q = r->q, P1 = std::max<int64_t>(P, 1);
  if ((e = dalloc(&r->Q, (size_t)(q * N))) || (e = dalloc(&r->Yres, (size_t)(P1 * N))) ||
      (e = dalloc(&r->s, (size_t)P1)) || (e = dalloc(&r->col_s, (size_t)P1)) ||
      (e = dalloc(&r->col_rmul, (size_t)Pp)) || (e = dalloc(&r->col_cs, (size_t)Pp)) ||
      (e = dalloc(&r->qcs, (size_t)QCOLS)) || (e = dalloc(&r->Bhi, (size_t)(Pp * Np))) ||
      (e = dalloc(&r->Blo, (size_t)(Pp * Np))) || (e = dalloc(&r->B32, (size_t)(Pp * Np))) ||
      (e = dalloc(&r->QB, (size_t)(QCOLS * Np))) || (e = dalloc(&r->QBhi, (size_t)(QCOLS * Np))) ||
      (e = dalloc(&r->QBlo, (size_t)(QCOLS * Np))) || (e = dalloc(&r->samples, (size_t)nw)))
    return cleanup(cuda_fail(e, "tg_prepare_panel_subset allocation"));
  auto run = [&]() -> cudaError_t {
    cudaError_t x;
    const int64_t Nc = pc->Npad;
    if ((x = cudaMemsetAsync(r->Q, 0, sizeof(double) * q * N, st)) ||
        (x = cudaMemsetAsync(r->Yres, 0, sizeof(double) * P1 * N, st)) ||
        (x = cudaMemsetAsync(r->Bhi, 0, 2 * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->Blo, 0, 2 * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->B32, 0, 4 * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->QB, 0, 4 * QCOLS * Np, st)) ||
        (x = cudaMemsetAsync(r->QBhi, 0, 2 * QCOLS * Np, st)) ||
        (x = cudaMemsetAsync(r->QBlo, 0, 2 * QCOLS * Np, st)))
      return x;
    if ((x = launch_scatter(pc->Q, NS, r->Q, N, didx, NS, q, 8, st)) ||
        (x = launch_scatter(pc->Yres, NS, r->Yres, N, didx, NS, P, 8, st)) ||
        (x = launch_scatter(pc->Bhi, Nc, r->Bhi, Np, didx, NS, Pp, 2, st)) ||
        (x = launch_scatter(pc->Blo, Nc, r->Blo, Np, didx, NS, Pp, 2, st)) ||
        (x = launch_scatter(pc->B32, Nc, r->B32, Np, didx, NS, Pp, 4, st)) ||
        (x = launch_scatter(pc->QB, Nc, r->QB, Np, didx, NS, QCOLS, 4, st)) ||
        (x = launch_scatter(pc->QBhi, Nc, r->QBhi, Np, didx, NS, QCOLS, 2, st)) ||
        (x = launch_scatter(pc->QBlo, Nc, r->QBlo, Np, didx, NS, QCOLS, 2, st)))
      return x;
    if ((x = cudaMemcpyAsync(r->s, pc->s, sizeof(double) * P1, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->col_s, pc->col_s, sizeof(float) * P1, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->col_rmul, pc->col_rmul, sizeof(float) * Pp, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->col_cs, pc->col_cs, sizeof(float) * Pp, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->qcs, pc->qcs, sizeof(float) * QCOLS, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->samples, hm.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, st)))
      return x;
    return cudaStreamSynchronize(st);
  };
  if ((e = run())) return cleanup(cuda_fail(e, "tg_prepare_panel_subset scatter"));
  if (N % 32) {  // bits past N are not samples
    const uint32_t last = hm[(size_t)(nw - 1)] & ((1u << (N % 32)) - 1u);
    if ((e = cudaMemcpy(r->samples + nw - 1, &last, sizeof(uint32_t), cudaMemcpyHostToDevice)))
      return cleanup(cuda_fail(e, "tg_prepare_panel_subset sample mask"));
  }
  if (!make_tmap(&r->tmBhi, r->Bhi, Pp, Np, Np, 256) || !make_tmap(&r->tmBlo, r->Blo, Pp, Np, Np, 256) ||
      !make_tmap(&r->tmBhi2, r->Bhi, Pp, Np, Np, 128) || !make_tmap(&r->tmBlo2, r->Blo, Pp, Np, Np, 128) ||
      !make_tmap(&r->tmQhi, r->QBhi, QCOLS, Np, Np, 64) || !make_tmap(&r->tmQlo, r->QBlo, QCOLS, Np, Np, 64) ||
      !make_tmap(&r->tmBhi64, r->Bhi, Pp, Np, Np, 64) || !make_tmap(&r->tmBlo64, r->Blo, Pp, Np, Np, 64))
    return cleanup(fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the subset panel"));
  const tg_status js = build_joint(r, st);
  if (js != TG_OK) return cleanup(js);
  tg_panel* done = r;
  r = nullptr;
  cleanup(TG_OK);
  *out = done;
  return TG_OK;
}

tg_status tg_panel_samples(const tg_panel* p, int64_t* n_used, const uint32_t** samples) {
  TG_ARG(p, "null panel");
  if (n_used) *n_used = p->NS;
  if (samples) *samples = p->samples;
  return TG_OK;
}

tg_status tg_phenotype_masks(tg_ctx* c, const float* Y, int64_t ldy, int64_t N, int64_t P,
                             uint32_t* masks, int64_t ldm, void* stream) {
  TG_ARG(c && N > 0 && P >= 0, "bad arguments");
  TG_ARG((Y && masks) || P == 0, "null Y or masks");
  TG_ARG(ldy >= N && ldm >= (N + 31) / 32, "ldy < N or ldm < ceil(N/32)");
  TG_CUDA(cudaSetDevice(c->device));
  TG_CUDA(launch_pheno_masks(Y, ldy, N, P, masks, ldm, (cudaStream_t)stream));
  return TG_OK;
}

tg_status tg_panel_info(const tg_panel* p, int64_t* N, int64_t* P, int64_t* q, int64_t* df) {
  TG_ARG(p, "null panel");
  if (N) *N = p->N;
  if (P) *P = p->P;
  if (q) *q = p->q;
  if (df) *df = p->df;
  return TG_OK;
}

tg_status tg_panel_Q(const tg_panel* p, const double** Q, int64_t* ldq, int64_t* q) {
  TG_ARG(p, "null panel");
  if (Q) *Q = p->Q;
  if (ldq) *ldq = p->N;
  if (q) *q = p->q;
  return TG_OK;
}

tg_status tg_panel_Yres(const tg_panel* p, const double** Yres, int64_t* ld, const double** s) {
  TG_ARG(p, "null panel");
  if (Yres) *Yres = p->Yres;
  if (ld) *ld = p->N;
  if (s) *s = p->s;
  return TG_OK;
}

tg_status tg_panel_free(tg_panel* p) {
  if (!p) return TG_OK;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  dfree(p->X); dfree(p->Q); dfree(p->Yres); dfree(p->s); dfree(p->col_s); dfree(p->col_rmul);
  dfree(p->col_cs); dfree(p->qcs); dfree(p->samples);
  dfree(p->Bhi); dfree(p->Blo); dfree(p->B32); dfree(p->QB); dfree(p->QBhi); dfree(p->QBlo);
  dfree(p->QYhi); dfree(p->QYlo); dfree(p->qycs);
  dfree(p->QYhi16); dfree(p->QYlo16); dfree(p->qycs16);
  dfree(p->QBhi16); dfree(p->QBlo16); dfree(p->qcs16);
  dfree(p->fp4B); dfree(p->fp4B_scale); dfree(p->fp4B_cs);
  dfree(p->fp4Q); dfree(p->fp4Q_scale); dfree(p->fp4Q_cs);
  delete p;
  return TG_OK;
}

tg_status tg_decode_block(tg_ctx* c, const uint8_t* G, int64_t ldg, int32_t encoding, int64_t N,
                          int64_t M, const uint32_t* missing, int64_t ldm, int32_t precision,
                          void* A, float* shift, int64_t lda, int32_t* n_obs, int64_t* S,
                          int64_t* S2, double* mean, void* stream) {
  TG_ARG(c, "null context");
  TG_ARG(encoding == TG_ENC_2BIT || encoding == TG_ENC_U8_DOSAGE, "unknown encoding");
  TG_ARG(precision == TG_PREC_FP32 || precision == TG_PREC_SPLIT_BF16, "unknown precision");
  TG_ARG(N > 0 && M >= 0, "bad sizes");
  if (M == 0) return TG_OK;
  TG_ARG(G && aligned(G, 16), "G must be a 16-byte aligned device pointer");
  const int64_t need = encoding == TG_ENC_2BIT ? (N + 3) / 4 : N;
  TG_ARG(ldg >= need && ldg % 16 == 0, "ldg must be >= the packed row length and a multiple of 16");
  if (encoding == TG_ENC_2BIT) TG_ARG(missing == nullptr, "missing must be NULL for 2-bit calls");
  if (missing) TG_ARG(ldm >= (N + 31) / 32, "ldm too small");
  TG_ARG(A && aligned(A, 16), "A must be a 16-byte aligned device pointer");
  TG_ARG(lda >= N && lda % KPAD == 0, "lda must be >= N and a multiple of 64");
  if (precision == TG_PREC_FP32) TG_ARG(shift == nullptr, "shift must be NULL for FP32");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  StageScope s(c, STAGE_DECODE, st, 1);
  TG_CUDA(launch_decode(G, ldg, encoding, N, M, missing, ldm, precision, A, shift, nullptr, lda,
                        n_obs, S, S2, mean, nullptr, st));
  return TG_OK;
}

tg_status tg_scan_block(tg_ctx* c, const tg_panel* p, const uint8_t* G, int64_t ldg,
                        int32_t encoding, int64_t N, int64_t M, int64_t marker_offset,
                        const uint32_t* missing, int64_t ldm, const tg_scan_opts* opts,
                        const tg_outputs* out, void* stream) {
  TG_ARG(opts && out, "null options or outputs");
  ScanArgs a{G, ldg, encoding, N, M, marker_offset, missing, ldm, *opts, *out};
  tg_status s = check_scan_args(c, p, a);
  if (s != TG_OK) return s;
  TG_CUDA(cudaSetDevice(c->device));
  return scan_impl(c, p, a, (cudaStream_t)stream);
}

// Largest block_markers of the host-streamed scan: keeps f * block sizes and block bytes far
// inside int64.
constexpr int64_t kMaxBlockMarkers = 1ll << 32;
// Alignment of each block's bytes in the host-streamed scan's device ring (that of cudaMalloc).
constexpr int64_t kRingAlign = 256;

// Block sizes of tg_scan_host for M markers (B <= kMaxBlockMarkers, f in [1, 8]):
// round_up(B / 8, 256) first when B >= 2048 (else B), each next one f times the previous
// rounded up to 256, at most B; the last takes the rest. Calls emit(rows) per block in order.
extern "C++" {
template <class Emit>
void for_each_host_block(int64_t M, int64_t B, double f, Emit emit) {
  int64_t next = B >= 8 * 256 ? round_up(B / 8, 256) : B;
  for (int64_t m0 = 0; m0 < M;) {
    const int64_t rows = std::min<int64_t>(next, M - m0);
    emit(rows);
    m0 += rows;
    next = std::min<int64_t>(B, round_up((int64_t)((double)next * f), 256));
  }
}
}

std::vector<int64_t> host_block_sizes(int64_t M, int64_t B, double f) {
  std::vector<int64_t> v;
  for_each_host_block(M, B, f, [&](int64_t rows) { v.push_back(rows); });
  return v;
}

tg_status tg_host_block_sizes(int64_t M, int64_t block_markers, double factor, int64_t* sizes,
                              int64_t capacity, int64_t* n_blocks) {
  TG_ARG(M >= 0 && block_markers > 0 && n_blocks, "bad arguments");
  TG_ARG(block_markers <= kMaxBlockMarkers, "block_markers above 2^32");
  TG_ARG(factor >= 1.0 && factor <= 8.0, "growth factor must be in [1, 8]");
  TG_ARG(capacity >= 0 && (sizes || capacity == 0), "bad size buffer");
  // blocks never shrink below the first one, which bounds their number
  const int64_t first = block_markers >= 8 * 256 ? round_up(block_markers / 8, 256) : block_markers;
  if (M / first >= (1ll << 28)) return fail(TG_ERR_UNSUPPORTED, "more than 2^28 blocks");
  int64_t n = 0;  // counted as they come: nothing is stored beyond the caller's capacity
  for_each_host_block(M, block_markers, factor, [&](int64_t rows) {
    if (n < capacity) sizes[n] = rows;
    ++n;
  });
  *n_blocks = n;
  return TG_OK;
}

// Growth factor of tg_scan_host's block sizes: fixed by the caller, else the last measured
// scan / copy ratio within [1, 2], else 2.
double host_ramp_factor(const tg_ctx* c) {
  if (c->ramp_fixed > 0.0) return c->ramp_fixed;
  return c->ramp_ratio > 0.0 ? std::min(2.0, std::max(1.0, c->ramp_ratio)) : 2.0;
}

tg_status tg_set_host_ramp(tg_ctx* c, double factor) {
  TG_ARG(c, "null context");
  TG_ARG(factor == 0.0 || (factor >= 1.0 && factor <= 8.0), "ramp factor must be 0 or in [1, 8]");
  c->ramp_fixed = factor;
  return TG_OK;
}

tg_status tg_set_host_buffers(tg_ctx* c, int n_buffers) {
  TG_ARG(c, "null context");
  TG_ARG(n_buffers >= 2 && n_buffers <= kMaxHostBufs, "host buffers must be 2, 3 or 4");
  TG_CUDA(cudaSetDevice(c->device));
  // tg_scan_host is synchronous: between calls no copy or scan uses the ring, which the next
  // call allocates again at the new size
  if (n_buffers != c->host_bufs) {
    dfree(c->stage);
    c->stage_cap = 0;
  }
  c->host_bufs = n_buffers;
  return TG_OK;
}

tg_status tg_host_ramp(const tg_ctx* c, double* factor, double* measured_ratio) {
  TG_ARG(c, "null context");
  if (factor) *factor = host_ramp_factor(c);
  if (measured_ratio) *measured_ratio = c->ramp_ratio;
  return TG_OK;
}

tg_status tg_scan_host(tg_ctx* c, const tg_panel* p, const uint8_t* G_host, int64_t ldg,
                       int32_t encoding, int64_t N, int64_t M, int64_t block_markers,
                       int64_t marker_offset, const tg_scan_opts* opts, tg_hit* hits_host,
                       int64_t hit_capacity, int64_t* n_hits, unsigned long long* best_host,
                       void* stream) {
  TG_ARG(c && p && opts && n_hits, "null argument");
  TG_ARG(!opts->full_output, "tg_scan_host collects hits only");
  TG_ARG(block_markers > 0 && M >= 0, "bad block size");
  TG_ARG(block_markers <= kMaxBlockMarkers, "block_markers above 2^32");
  TG_ARG(ldg > 0 && ldg <= (1ll << 31), "bad ldg");
  TG_ARG(hit_capacity >= 0 && (hits_host || hit_capacity == 0), "bad hit buffer");
  TG_ARG(G_host || M == 0, "null G_host");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  // the ring: host_bufs whole blocks, each starting on a 256-byte boundary
  const size_t blk_bytes = (size_t)round_up(block_markers * ldg, kRingAlign);
  const size_t ring_bytes = blk_bytes * (size_t)c->host_bufs;
  if (c->stage_cap < ring_bytes) {  // larger blocks: a new ring
    dfree(c->stage);
    c->stage_cap = 0;
    TG_CUDA(dalloc(&c->stage, ring_bytes));
    c->stage_cap = ring_bytes;
  }
  if (c->dhits_cap < std::max<int64_t>(hit_capacity, 1)) {
    dfree(c->dhits);
    c->dhits_cap = 0;
    TG_CUDA(dalloc(&c->dhits, (size_t)std::max<int64_t>(hit_capacity, 1)));
    c->dhits_cap = std::max<int64_t>(hit_capacity, 1);
  }
  if (!c->dnhits) TG_CUDA(dalloc(&c->dnhits, 1));
  if (c->dbest_cap < p->P) {
    dfree(c->dbest);
    c->dbest_cap = 0;
    TG_CUDA(dalloc(&c->dbest, (size_t)std::max<int64_t>(p->P, 1)));
    c->dbest_cap = p->P;
  }
  TG_CUDA(cudaMemsetAsync(c->dnhits, 0, sizeof(unsigned long long), st));
  TG_CUDA(cudaMemsetAsync(c->dbest, 0, sizeof(unsigned long long) * (size_t)std::max<int64_t>(p->P, 1), st));
  tg_outputs o{};
  o.hits = c->dhits;
  o.hit_capacity = hit_capacity;
  o.n_hits = c->dnhits;
  o.best = best_host ? c->dbest : nullptr;
  // Block sizes ramp up from about block_markers / 8 by a factor f per block, so that only a
  // short first copy runs before the first scan, and each copy hides behind the previous
  // block's scan as long as it is at most f times shorter. f = 2 until a call has timed the
  // scans of its second to ninth blocks against their copies; then f is the ratio of the sums
  // within [1, 2]: with copies about as slow as the scans, larger blocks would only leave the
  // scan waiting for their copies. (Several blocks, because one copy's rate varies.)
  const std::vector<int64_t> sizes = host_block_sizes(M, block_markers, host_ramp_factor(c));
  int64_t timed = 0;  // blocks timed (1 .. kRateBlocks)
  // Blocks fill the ring front to back, each at the next 256-byte boundary, and wrap to its
  // start when the next one does not fit before the end. A block's copy waits (on the side
  // stream) for the scans of the earlier blocks whose bytes it overwrites; the scans finish in
  // order on `stream`, so waiting for the newest of them is enough. The ramped first blocks are
  // smaller than block_markers, so up to 8 x host_bufs of them are in flight at once: the copies
  // run as far ahead of the scans as the ring's bytes allow, which absorbs a host link whose
  // rate varies from copy to copy.
  struct InFlight {
    size_t off, end;
    int ev;
  };
  std::vector<InFlight> q;  // blocks whose scan may still read their bytes, oldest first
  size_t head = 0, q0 = 0;  // q0: first live entry of q
  for (int64_t m0 = 0, b = 0, rows = 0; b < (int64_t)sizes.size(); m0 += rows, ++b) {
    rows = sizes[(size_t)b];
    const size_t len = (size_t)(rows * ldg);
    size_t off = (size_t)round_up((int64_t)head, kRingAlign);
    if (off + len > c->stage_cap) off = 0;
    // the newest live block that overlaps [off, off + len); at least enough of the oldest to
    // keep fewer than kRingEvents live, so that this block's event is not still awaited
    int64_t last = -1;
    for (size_t j = q0; j < q.size(); ++j)
      if (q[j].off < off + len && off < q[j].end) last = (int64_t)j;
    const int64_t live = (int64_t)(q.size() - q0);
    if (live >= kRingEvents) last = std::max<int64_t>(last, (int64_t)q0 + live - kRingEvents);
    if (last >= 0) {
      TG_CUDA(cudaStreamWaitEvent(c->side, c->ev_free[q[(size_t)last].ev], 0));
      q0 = (size_t)last + 1;
    }
    uint8_t* dst = c->stage + off;
    // blocks 1 .. kRateBlocks: their copies and scans, each timed on its own stream
    const bool time_it = b >= 1 && b <= kRateBlocks;
    cudaEvent_t* er = c->ev_rate + 4 * (b - 1);
    if (time_it) TG_CUDA(cudaEventRecord(er[0], c->side));
    {
      StageScope s(c, STAGE_H2D, c->side, 0);
      TG_CUDA(cudaMemcpyAsync(dst, G_host + m0 * ldg, len, cudaMemcpyHostToDevice, c->side));
    }
    if (time_it) TG_CUDA(cudaEventRecord(er[1], c->side));
    // a wait takes the event's latest record at the time of the call: one event serves all
    TG_CUDA(cudaEventRecord(c->ev_copied, c->side));
    TG_CUDA(cudaStreamWaitEvent(st, c->ev_copied, 0));
    if (time_it) TG_CUDA(cudaEventRecord(er[2], st));
    ScanArgs a{dst, ldg, encoding, N, rows, marker_offset + m0, nullptr, 0, *opts, o};
    tg_status s = check_scan_args(c, p, a);
    if (s != TG_OK) return s;
    s = scan_impl(c, p, a, st);
    if (s != TG_OK) return s;
    if (time_it) {
      TG_CUDA(cudaEventRecord(er[3], st));
      timed = b;
    }
    const int ev = (int)(b % kRingEvents);
    TG_CUDA(cudaEventRecord(c->ev_free[ev], st));
    q.push_back({off, off + len, ev});
    head = off + len;
  }
  unsigned long long nh = 0;
  TG_CUDA(cudaMemcpyAsync(&nh, c->dnhits, sizeof(nh), cudaMemcpyDeviceToHost, st));
  TG_CUDA(cudaStreamSynchronize(st));
  *n_hits = (int64_t)nh;
  const int64_t ncopy = std::min<int64_t>((int64_t)nh, hit_capacity);
  if (ncopy > 0)
    TG_CUDA(cudaMemcpyAsync(hits_host, c->dhits, sizeof(tg_hit) * (size_t)ncopy,
                            cudaMemcpyDeviceToHost, st));
  if (best_host)
    TG_CUDA(cudaMemcpyAsync(best_host, c->dbest, sizeof(unsigned long long) * (size_t)p->P,
                            cudaMemcpyDeviceToHost, st));
  TG_CUDA(cudaStreamSynchronize(st));
  if (timed > 0) {  // both streams are past the timed blocks: every scan has finished
    double copy_ms = 0.0, scan_ms = 0.0;
    bool ok = true;
    for (int64_t i = 0; i < timed && ok; ++i) {
      float cm = 0.0f, sm = 0.0f;
      ok = cudaEventElapsedTime(&cm, c->ev_rate[4 * i], c->ev_rate[4 * i + 1]) == cudaSuccess &&
           cudaEventElapsedTime(&sm, c->ev_rate[4 * i + 2], c->ev_rate[4 * i + 3]) == cudaSuccess;
      copy_ms += cm;
      scan_ms += sm;
    }
    if (ok && copy_ms > 0.0) c->ramp_ratio = scan_ms / copy_ms;
  }
  // synchronous, so the call reports what its kernels latched, and leaves the word clear
  uint32_t word = 0;
  TG_CUDA(cudaMemcpy(&word, c->status, sizeof(word), cudaMemcpyDeviceToHost));
  TG_CUDA(cudaMemset(c->status, 0, sizeof(word)));
  if (word & ST_TIMEOUT) return fail(TG_ERR_TIMEOUT, "a bounded device wait ran out");
  if ((int64_t)nh > hit_capacity || (word & ST_CAPACITY))
    return fail(TG_ERR_CAPACITY, "more hits than hit_capacity");
  return TG_OK;
}

tg_status tg_status_poll(tg_ctx* c, void* stream) {
  TG_ARG(c, "null context");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t word = 0;
  TG_CUDA(cudaStreamSynchronize(st));
  TG_CUDA(cudaMemcpy(&word, c->status, sizeof(word), cudaMemcpyDeviceToHost));
  TG_CUDA(cudaMemset(c->status, 0, sizeof(word)));
  if (word & ST_TIMEOUT) return fail(TG_ERR_TIMEOUT, "a bounded device wait ran out");
  if (word & ST_CAPACITY) return fail(TG_ERR_CAPACITY, "more hits than hit_capacity");
  return TG_OK;
}

tg_status tg_set_fused_decode(tg_ctx* c, int enable) {
  TG_ARG(c, "null context");
  TG_ARG(enable >= 0 && enable <= 2, "fused decode setting must be 0, 1 or 2");
  TG_ARG(c->graphs_alive == 0, "a captured scan graph uses this context");
  c->fuse_decode = enable == 1;
  c->fuse_joint = enable != 0;
  return TG_OK;
}

tg_status tg_set_profiling(tg_ctx* c, int enable) {
  TG_ARG(c, "null context");
  c->prof = enable != 0;
  return TG_OK;
}

tg_status tg_stage_times(tg_ctx* c, double* ms, int64_t* launches, int reset) {
  TG_ARG(c, "null context");
  TG_CUDA(cudaSetDevice(c->device));
  for (auto& ev : c->pending) {
    TG_CUDA(cudaEventSynchronize(ev.b));
    float t = 0.f;
    TG_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
    c->stage_ms[ev.stage] += t;
    c->event_pool.push_back(ev.a);
    c->event_pool.push_back(ev.b);
  }
  c->pending.clear();
  for (int i = 0; i < TG_N_STAGES; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->launches[i];
    if (reset) {
      c->stage_ms[i] = 0;
      c->launches[i] = 0;
    }
  }
  return TG_OK;
}

tg_status tg_bounded_wait_test(tg_ctx* c, const uint32_t* flag, int64_t limit_ns, void* stream) {
  TG_ARG(c && flag && limit_ns > 0, "bad argument");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* res = c->scratch + 8;
  TG_CUDA(cudaMemsetAsync(res, 0, sizeof(uint32_t), st));
  TG_CUDA(launch_wait_test(flag, limit_ns, res, st));
  uint32_t h = 0;
  TG_CUDA(cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
  TG_CUDA(cudaStreamSynchronize(st));
  if (h == 2u) return fail(TG_ERR_TIMEOUT, "the flag was not set within the limit");
  if (h != 1u) return fail(TG_ERR_CUDA, "wait kernel did not report");
  return TG_OK;
}


// ------------------------------------------------------------------ batched form

tg_status tg_panel_concat(tg_ctx* c, const tg_panel* const* panels, int n, tg_panel** out,
                          void* stream) {
  TG_ARG(c && panels && out && n >= 1, "bad arguments");
  *out = nullptr;
  const tg_panel* p0 = panels[0];
  TG_ARG(p0 != nullptr, "null panel");
  int64_t P = 0;
  for (int i = 0; i < n; ++i) {
    TG_ARG(panels[i] != nullptr, "null panel");
    const tg_panel* pi = panels[i];
    TG_ARG(pi->N == p0->N && pi->NS == p0->NS && pi->q == p0->q && pi->n_cov == p0->n_cov &&
               pi->device == p0->device && (pi->samples != nullptr) == (p0->samples != nullptr),
           "panels differ in samples or covariate rank");
    P += pi->P;
  }
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = p0->N, q = p0->q;
  // the covariate bases must be identical (same covariates, same deterministic QR)
  {
    std::vector<double> a((size_t)(q * N)), b((size_t)(q * N));
    TG_CUDA(cudaMemcpy(a.data(), p0->Q, sizeof(double) * a.size(), cudaMemcpyDeviceToHost));
    for (int i = 1; i < n; ++i) {
      TG_CUDA(cudaMemcpy(b.data(), panels[i]->Q, sizeof(double) * b.size(), cudaMemcpyDeviceToHost));
      if (std::memcmp(a.data(), b.data(), sizeof(double) * a.size()) != 0)
        return fail(TG_ERR_INVALID_ARG, "panels were prepared with different covariates");
    }
  }
  const int64_t nw = (N + 31) / 32;
  std::vector<uint32_t> mask0;
  if (p0->samples) {  // subset panels: the same samples
    mask0.resize((size_t)nw);
    std::vector<uint32_t> mi((size_t)nw);
    TG_CUDA(cudaMemcpy(mask0.data(), p0->samples, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost));
    for (int i = 1; i < n; ++i) {
      TG_CUDA(cudaMemcpy(mi.data(), panels[i]->samples, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost));
      if (mi != mask0) return fail(TG_ERR_INVALID_ARG, "subset panels use different samples");
    }
  }
  tg_panel* r = new tg_panel();
  r->device = p0->device;
  r->N = N;
  r->P = P;
  r->n_cov = p0->n_cov;
  r->q = q;
  r->df = p0->df;
  r->Npad = p0->Npad;
  r->Ppad = round_up(std::max<int64_t>(P, 1), PPAD);
  r->lnB = p0->lnB;
  r->lnB_paper = p0->lnB_paper;
  r->NS = p0->NS;
  const int64_t Np = r->Npad, Pp = r->Ppad;
  cudaError_t e;
  if (!mask0.empty()) {
    if ((e = dalloc(&r->samples, (size_t)nw)) ||
        (e = cudaMemcpy(r->samples, mask0.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice))) {
      tg_panel_free(r);
      return cuda_fail(e, "tg_panel_concat allocation");
    }
  }
  if ((e = dalloc(&r->Q, (size_t)(q * N))) || (e = dalloc(&r->Yres, (size_t)(std::max<int64_t>(P, 1) * N))) ||
      (e = dalloc(&r->s, (size_t)std::max<int64_t>(P, 1))) ||
      (e = dalloc(&r->col_s, (size_t)std::max<int64_t>(P, 1))) || (e = dalloc(&r->col_rmul, (size_t)Pp)) ||
      (e = dalloc(&r->col_cs, (size_t)Pp)) || (e = dalloc(&r->qcs, (size_t)QCOLS)) ||
      (e = dalloc(&r->Bhi, (size_t)(Pp * Np))) || (e = dalloc(&r->Blo, (size_t)(Pp * Np))) ||
      (e = dalloc(&r->B32, (size_t)(Pp * Np))) || (e = dalloc(&r->QB, (size_t)(QCOLS * Np))) ||
      (e = dalloc(&r->QBhi, (size_t)(QCOLS * Np))) || (e = dalloc(&r->QBlo, (size_t)(QCOLS * Np)))) {
    tg_panel_free(r);
    return cuda_fail(e, "tg_panel_concat allocation");
  }
  auto run = [&]() -> cudaError_t {
    cudaError_t x;
    if ((x = cudaMemsetAsync(r->Bhi, 0, sizeof(__nv_bfloat16) * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->Blo, 0, sizeof(__nv_bfloat16) * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->B32, 0, sizeof(float) * Pp * Np, st)) ||
        (x = cudaMemsetAsync(r->col_rmul, 0, sizeof(float) * Pp, st)) ||
        (x = cudaMemsetAsync(r->col_cs, 0, sizeof(float) * Pp, st)) ||
        (x = cudaMemcpyAsync(r->qcs, p0->qcs, sizeof(float) * QCOLS, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->Q, p0->Q, sizeof(double) * q * N, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->QB, p0->QB, sizeof(float) * QCOLS * Np, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->QBhi, p0->QBhi, 2 * QCOLS * Np, cudaMemcpyDeviceToDevice, st)) ||
        (x = cudaMemcpyAsync(r->QBlo, p0->QBlo, 2 * QCOLS * Np, cudaMemcpyDeviceToDevice, st)))
      return x;
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
      const tg_panel* pi = panels[i];
      const int64_t k = pi->P;
      if (k == 0) continue;
      if ((x = cudaMemcpyAsync(r->Yres + off * N, pi->Yres, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->s + off, pi->s, sizeof(double) * k, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->col_s + off, pi->col_s, sizeof(float) * k, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->col_rmul + off, pi->col_rmul, sizeof(float) * k, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->col_cs + off, pi->col_cs, sizeof(float) * k, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->Bhi + off * Np, pi->Bhi, 2 * k * Np, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->Blo + off * Np, pi->Blo, 2 * k * Np, cudaMemcpyDeviceToDevice, st)) ||
          (x = cudaMemcpyAsync(r->B32 + off * Np, pi->B32, sizeof(float) * k * Np, cudaMemcpyDeviceToDevice, st)))
        return x;
      off += k;
    }
    return cudaStreamSynchronize(st);
  };
  if ((e = run())) {
    tg_panel_free(r);
    return cuda_fail(e, "tg_panel_concat copy");
  }
  if (!make_tmap(&r->tmBhi, r->Bhi, Pp, Np, Np, 256) || !make_tmap(&r->tmBlo, r->Blo, Pp, Np, Np, 256) ||
      !make_tmap(&r->tmBhi2, r->Bhi, Pp, Np, Np, 128) || !make_tmap(&r->tmBlo2, r->Blo, Pp, Np, Np, 128) ||
      !make_tmap(&r->tmQhi, r->QBhi, QCOLS, Np, Np, 64) || !make_tmap(&r->tmQlo, r->QBlo, QCOLS, Np, Np, 64) ||
      !make_tmap(&r->tmBhi64, r->Bhi, Pp, Np, Np, 64) || !make_tmap(&r->tmBlo64, r->Blo, Pp, Np, Np, 64)) {
    tg_panel_free(r);
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the concatenated panel");
  }
  const tg_status js = build_joint(r, st);
  if (js != TG_OK) {
    tg_panel_free(r);
    return js;
  }
  *out = r;
  return TG_OK;
}

tg_status tg_scan_graph_create(tg_ctx* c, const tg_panel* p, int n_blocks,
                               const uint8_t* const* G, const int64_t* M,
                               const int64_t* marker_offset, const uint32_t* const* missing,
                               int64_t ldg, int64_t ldm, int32_t encoding, int64_t N,
                               const tg_scan_opts* opts, const tg_outputs* out, tg_graph** graph) {
  TG_ARG(c && p && G && M && marker_offset && opts && out && graph && n_blocks >= 1, "bad arguments");
  *graph = nullptr;
  if (opts->precision == TG_PREC_FP4_PIECES)
    return fail(TG_ERR_UNSUPPORTED, "the FP4 form is not captured in scan graphs");
  TG_ARG(!opts->full_output, "captured scan graphs collect hits and best markers only");
  TG_ARG(!out->marker_norm2 && !out->marker_nobs && !out->marker_mean,
         "per-marker outputs are not supported in captured scan graphs");
  TG_CUDA(cudaSetDevice(c->device));
  int64_t maxM = 0;
  for (int b = 0; b < n_blocks; ++b) {
    ScanArgs a{G[b], ldg, encoding, N, M[b], marker_offset[b], missing ? missing[b] : nullptr, ldm,
               *opts, *out};
    tg_status s = check_scan_args(c, p, a);
    if (s != TG_OK) return s;
    maxM = std::max(maxM, M[b]);
  }
  // size the workspace now: nothing may allocate inside the capture
  bool need_operand = opts->precision != TG_PREC_SPLIT_BF16 || !c->fuse_decode;
  for (int b = 0; b < n_blocks; ++b) need_operand |= missing && missing[b];
  {
    tg_status ws = reserve_graph_workspace(c, p, n_blocks, M, maxM, need_operand, *opts);
    if (ws != TG_OK) return ws;
  }
  cudaStream_t cap = nullptr;
  TG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  tg_graph* g = new tg_graph();
  g->ctx = c;
  int64_t before[TG_N_STAGES];
  std::memcpy(before, c->launches, sizeof(before));
  const bool prof = c->prof;
  c->prof = false;
  tg_status s = TG_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int b = 0; b < n_blocks && s == TG_OK; ++b) {
      ScanArgs a{G[b], ldg, encoding, N, M[b], marker_offset[b], missing ? missing[b] : nullptr,
                 ldm, *opts, *out};
      s = scan_impl(c, p, a, cap);
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
    if (e == cudaSuccess) e = e2;
  }
  c->prof = prof;
  for (int i = 0; i < TG_N_STAGES; ++i) {
    g->launches[i] = c->launches[i] - before[i];
    c->launches[i] = before[i];
  }
  cudaStreamDestroy(cap);
  if (s == TG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (s != TG_OK || e != cudaSuccess) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return s != TG_OK ? s : cuda_fail(e, "tg_scan_graph_create capture");
  }
  c->graphs_alive += 1;
  *graph = g;
  return TG_OK;
}

tg_status tg_scan_graph_create_host(tg_ctx* c, const tg_panel* p, int n_blocks,
                                    const uint8_t* const* G_host, const int64_t* M,
                                    const int64_t* marker_offset, int64_t ldg, int32_t encoding,
                                    int64_t N, const tg_scan_opts* opts, const tg_outputs* out,
                                    tg_graph** graph) {
  TG_ARG(c && p && G_host && M && marker_offset && opts && out && graph && n_blocks >= 1,
         "bad arguments");
  *graph = nullptr;
  if (opts->precision == TG_PREC_FP4_PIECES)
    return fail(TG_ERR_UNSUPPORTED, "the FP4 form is not captured in scan graphs");
  TG_ARG(!opts->full_output, "captured scan graphs collect hits and best markers only");
  TG_ARG(!out->marker_norm2 && !out->marker_nobs && !out->marker_mean,
         "per-marker outputs are not supported in captured scan graphs");
  TG_CUDA(cudaSetDevice(c->device));
  int64_t maxM = 0;
  for (int b = 0; b < n_blocks; ++b) {
    TG_ARG(M[b] == 0 || G_host[b] != nullptr, "null host block");
    // the arguments of the scan as it will run, from a device staging buffer
    ScanArgs a{reinterpret_cast<const uint8_t*>(uintptr_t(256)), ldg, encoding, N, M[b],
               marker_offset[b], nullptr, 0, *opts, *out};
    tg_status s = check_scan_args(c, p, a);
    if (s != TG_OK) return s;
    maxM = std::max(maxM, M[b]);
  }
  const bool need_operand = opts->precision != TG_PREC_SPLIT_BF16 || !c->fuse_decode;
  {
    tg_status ws = reserve_graph_workspace(c, p, n_blocks, M, maxM, need_operand, *opts);
    if (ws != TG_OK) return ws;
  }
  tg_graph* g = new tg_graph();
  g->ctx = c;
  const size_t blk_bytes = (size_t)std::max<int64_t>(maxM, 1) * (size_t)ldg;
  cudaStream_t cap = nullptr, side = nullptr;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // ev: 0 fork, 1 join, 2-3 block copied into staging buffer 0/1, 4-5 buffer 0/1 free again
  auto release = [&](tg_status s) {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
    if (cap) cudaStreamDestroy(cap);
    if (s != TG_OK) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      if (g->graph) cudaGraphDestroy(g->graph);
      dfree(g->stage[0]);
      dfree(g->stage[1]);
      delete g;
    }
    return s;
  };
  cudaError_t e;
  if ((e = dalloc(&g->stage[0], blk_bytes)) || (e = dalloc(&g->stage[1], blk_bytes)) ||
      (e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) ||
      (e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)))
    return release(cuda_fail(e, "tg_scan_graph_create_host set-up"));
  for (auto& x : ev)
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)))
      return release(cuda_fail(e, "tg_scan_graph_create_host events"));
  int64_t before[TG_N_STAGES];
  std::memcpy(before, c->launches, sizeof(before));
  const bool prof = c->prof;
  c->prof = false;
  tg_status s = TG_OK;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    auto step = [&]() -> tg_status {
      // the copy stream joins the capture, then every block: copy (side) -> scan (cap)
      TG_CUDA(cudaEventRecord(ev[0], cap));
      TG_CUDA(cudaStreamWaitEvent(side, ev[0], 0));
      bool used[2] = {false, false};
      for (int b = 0, nb = 0; b < n_blocks; ++b) {
        if (M[b] == 0) continue;
        const int buf = (nb++) & 1;
        if (used[buf]) TG_CUDA(cudaStreamWaitEvent(side, ev[4 + buf], 0));  // its last scan is done
        used[buf] = true;
        TG_CUDA(cudaMemcpyAsync(g->stage[buf], G_host[b], (size_t)M[b] * (size_t)ldg,
                                cudaMemcpyHostToDevice, side));
        TG_CUDA(cudaEventRecord(ev[2 + buf], side));
        TG_CUDA(cudaStreamWaitEvent(cap, ev[2 + buf], 0));
        ScanArgs a{g->stage[buf], ldg, encoding, N, M[b], marker_offset[b], nullptr, 0, *opts,
                   *out};
        tg_status r = scan_impl(c, p, a, cap);
        if (r != TG_OK) return r;
        TG_CUDA(cudaEventRecord(ev[4 + buf], cap));
      }
      TG_CUDA(cudaEventRecord(ev[1], side));  // the copy stream rejoins before the capture ends
      TG_CUDA(cudaStreamWaitEvent(cap, ev[1], 0));
      return TG_OK;
    };
    s = step();
    cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
    if (s == TG_OK && e2 != cudaSuccess) s = cuda_fail(e2, "tg_scan_graph_create_host capture");
  } else {
    s = cuda_fail(e, "tg_scan_graph_create_host capture");
  }
  c->prof = prof;
  for (int i = 0; i < TG_N_STAGES; ++i) {
    g->launches[i] = c->launches[i] - before[i];
    c->launches[i] = before[i];
  }
  if (s == TG_OK && (e = cudaGraphInstantiate(&g->exec, g->graph, 0)))
    s = cuda_fail(e, "tg_scan_graph_create_host instantiate");
  if (s != TG_OK) return release(s);
  c->graphs_alive += 1;
  *graph = g;
  return release(TG_OK);
}

tg_status tg_scan_graph_launch(tg_graph* g, void* stream) {
  TG_ARG(g && g->exec, "null graph");
  TG_CUDA(cudaSetDevice(g->ctx->device));
  TG_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  for (int i = 0; i < TG_N_STAGES; ++i) g->ctx->launches[i] += g->launches[i];
  return TG_OK;
}

tg_status tg_scan_graph_free(tg_graph* g) {
  if (!g) return TG_OK;
  cudaSetDevice(g->ctx->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->stage[0] || g->stage[1]) {
    cudaDeviceSynchronize();  // a replay may still read the staging buffers
    dfree(g->stage[0]);
    dfree(g->stage[1]);
  }
  g->ctx->graphs_alive -= 1;
  delete g;
  return TG_OK;
}

tg_status tg_autotune(tg_ctx* c, const tg_panel* p, int32_t encoding, int64_t M, void* stream) {
  TG_ARG(c && p && M > 0, "bad arguments");
  TG_ARG(encoding == TG_ENC_2BIT || encoding == TG_ENC_U8_DOSAGE, "unknown encoding");
  TG_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ldg = round_up(encoding == TG_ENC_2BIT ? (p->N + 3) / 4 : p->N, 16);
  uint8_t* G = nullptr;
  tg_hit* hits = nullptr;
  unsigned long long* cnt = nullptr;
  unsigned long long* best = nullptr;
  cudaError_t e;
  auto cleanup = [&]() { dfree(G); dfree(hits); dfree(cnt); dfree(best); };
  // chance hits of the random trial block (about 5e-8 of M x P tests per scan) stay far below
  // the trial capacity, so the trials never latch a capacity error in the context's status
  constexpr int64_t kTrialHits = 1 << 16;
  if ((e = dalloc(&G, (size_t)(M * ldg))) || (e = dalloc(&hits, kTrialHits)) || (e = dalloc(&cnt, 1)) ||
      (e = dalloc(&best, (size_t)std::max<int64_t>(p->P, 1)))) {
    cleanup();
    return cuda_fail(e, "tg_autotune allocation");
  }
  if ((e = launch_fill_random(G, (size_t)(M * ldg), 0x5eed5eedull, st)) ||
      (e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st)) ||
      (e = cudaMemsetAsync(best, 0, sizeof(unsigned long long) * (size_t)std::max<int64_t>(p->P, 1), st))) {
    cleanup();
    return cuda_fail(e, "tg_autotune fill");
  }
  tg_outputs o{};
  o.hits = hits;
  o.hit_capacity = kTrialHits;
  o.n_hits = cnt;
  o.best = best;
  const tg_scan_opts opts{TG_PREC_SPLIT_BF16, 0, 7.30103};
  ScanArgs a{G, ldg, encoding, p->N, M, 0, nullptr, 0, opts, o};
  const int b = tune_bucket(M);
  // kernel, raster group, split-K (the one-CTA kernel splits K when its tiles are fewer than
  // the SMs; panels of at most 64 phenotypes take 64-column tiles whatever the choice)
  const int kinds[] = {TUNE_PAIR, TUNE_PAIR, TUNE_PAIR, TUNE_PAIR, TUNE_SINGLE, TUNE_SINGLE,
                       TUNE_SINGLE, TUNE_SINGLE, TUNE_SINGLE};
  const int groups[] = {4, 8, 16, 32, 8, 16, 32, 16, 16};
  const int splits[] = {1, 1, 1, 1, 1, 1, 1, 2, 4};
  const int64_t single_tiles = ((M + MT - 1) / MT) * ((p->P + 255) / 256);
  const int n_cand = p->P > 64 && single_tiles * 2 <= c->sm_count ? 9 : 7;
  const int save_k = c->tune_kernel[b], save_g = c->tune_group[b], save_s = c->tune_split[b];
  const bool prof = c->prof;
  // the trial launches do not count in the caller's stage statistics
  tg_stage_times(c, nullptr, nullptr, 0);
  double save_ms[TG_N_STAGES];
  int64_t save_n[TG_N_STAGES];
  std::memcpy(save_ms, c->stage_ms, sizeof(save_ms));
  std::memcpy(save_n, c->launches, sizeof(save_n));
  double best_ms = 1e30;
  int best_i = -1;
  tg_status s = TG_OK;
  for (int i = 0; i < n_cand && s == TG_OK; ++i) {
    c->tune_kernel[b] = kinds[i];
    c->tune_group[b] = groups[i];
    c->tune_split[b] = splits[i];
    c->prof = false;
    s = scan_impl(c, p, a, st);  // warm-up (and first-use set-up)
    if (s != TG_OK) break;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st))) { s = cuda_fail(e, "autotune"); break; }
    double ms_before[TG_N_STAGES];
    int64_t n_before[TG_N_STAGES];
    tg_stage_times(c, ms_before, n_before, 0);
    c->prof = true;
    for (int r = 0; r < 2 && s == TG_OK; ++r) {
      if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st))) { s = cuda_fail(e, "autotune"); break; }
      s = scan_impl(c, p, a, st);
    }
    c->prof = false;
    double ms_after[TG_N_STAGES];
    int64_t n_after[TG_N_STAGES];
    tg_stage_times(c, ms_after, n_after, 0);
    const double t = (ms_after[STAGE_GEMM] - ms_before[STAGE_GEMM]) / 2.0;
    if (t < best_ms) {
      best_ms = t;
      best_i = i;
    }
  }
  c->prof = prof;
  if (s == TG_OK) {
    if ((e = cudaStreamSynchronize(st))) s = cuda_fail(e, "tg_autotune");
  }
  tg_stage_times(c, nullptr, nullptr, 0);
  std::memcpy(c->stage_ms, save_ms, sizeof(save_ms));
  std::memcpy(c->launches, save_n, sizeof(save_n));
  if (s != TG_OK || best_i < 0) {
    c->tune_kernel[b] = save_k;
    c->tune_group[b] = save_g;
    c->tune_split[b] = save_s;
  } else {
    c->tune_kernel[b] = kinds[best_i];
    c->tune_group[b] = groups[best_i];
    c->tune_split[b] = splits[best_i];
  }
  cleanup();
  return s;
}

tg_status tg_set_tuning(tg_ctx* c, int64_t M, int32_t kernel, int32_t group) {
  TG_ARG(c && M > 0, "bad arguments");
  TG_ARG(kernel == 1 || kernel == 2, "kernel must be 1 (one CTA per tile) or 2 (CTA pairs)");
  TG_ARG(group >= 1 && group <= 1024, "group must be in [1, 1024]");
  const int b = tune_bucket(M);
  c->tune_kernel[b] = kernel == 1 ? TUNE_SINGLE : TUNE_PAIR;
  c->tune_group[b] = group;
  return TG_OK;
}

tg_status tg_set_tuning_split(tg_ctx* c, int64_t M, int32_t splits) {
  TG_ARG(c && M > 0, "bad arguments");
  TG_ARG(splits == 1 || splits == 2 || splits == 4, "splits must be 1, 2 or 4");
  c->tune_split[tune_bucket(M)] = splits;
  return TG_OK;
}

tg_status tg_tuning_split(const tg_ctx* c, int64_t M, int32_t* splits) {
  TG_ARG(c && M > 0 && splits, "bad arguments");
  const int t = c->tune_split[tune_bucket(M)];
  *splits = t > 1 ? t : 1;
  return TG_OK;
}

tg_status tg_tuning_save(const tg_ctx* c, const char* path) {
  TG_ARG(c && path, "null context or path");
  std::string j = "{\"format\": \"tg-tuning\", \"version\": 1, \"buckets\": [";
  bool first = true;
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (c->tune_kernel[b] == TUNE_DEFAULT) continue;
    char line[192];
    std::snprintf(line, sizeof(line),
                  "%s\n  {\"min_markers\": %lld, \"kernel\": \"%s\", \"group_m\": %d, "
                  "\"splits\": %d}",
                  first ? "" : ",", 1ll << b, c->tune_kernel[b] == TUNE_SINGLE ? "single" : "pair",
                  c->tune_group[b] > 0 ? c->tune_group[b] : kGroupDefault,
                  c->tune_split[b] > 1 ? c->tune_split[b] : 1);
    j += line;
    first = false;
  }
  j += "\n]}\n";
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(TG_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const bool ok = std::fwrite(j.data(), 1, j.size(), f) == j.size();
  if (std::fclose(f) != 0 || !ok) return fail(TG_ERR_INVALID_ARG, std::string("cannot write ") + path);
  return TG_OK;
}

tg_status tg_tuning_load(tg_ctx* c, const char* path) {
  TG_ARG(c && path, "null context or path");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(TG_ERR_INVALID_ARG, std::string("cannot read ") + path);
  std::string j;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) j.append(buf, n);
  std::fclose(f);
  if (j.find("\"tg-tuning\"") == std::string::npos)
    return fail(TG_ERR_INVALID_ARG, "not a tuning file written by tg_tuning_save");
  // every entry first, then applied together, so that a bad file changes nothing
  int kern[kTuneBuckets], grp[kTuneBuckets], spl[kTuneBuckets];
  std::memcpy(kern, c->tune_kernel, sizeof(kern));
  std::memcpy(grp, c->tune_group, sizeof(grp));
  std::memcpy(spl, c->tune_split, sizeof(spl));
  // the integer after "key": in one entry; false if absent or not a number
  auto num_in = [](const std::string& e, const char* key, long long* v) -> bool {
    const size_t k = e.find(key);
    if (k == std::string::npos) return false;
    const size_t colon = e.find(':', k);
    if (colon == std::string::npos) return false;
    const char* start = e.c_str() + colon + 1;
    char* end = nullptr;
    *v = std::strtoll(start, &end, 10);
    return end != start;
  };
  size_t pos = j.find('[');
  int entries = 0;
  while (pos != std::string::npos && (pos = j.find('{', pos + 1)) != std::string::npos) {
    const size_t close = j.find('}', pos);
    if (close == std::string::npos) break;
    const std::string e = j.substr(pos, close - pos + 1);
    long long mm = 0, gm = 0, sp = 0;
    const bool single = e.find("\"single\"") != std::string::npos;
    const bool pair = e.find("\"pair\"") != std::string::npos;
    if (!num_in(e, "\"min_markers\"", &mm) || !num_in(e, "\"group_m\"", &gm) ||
        !num_in(e, "\"splits\"", &sp) || single == pair || mm < 1 || gm < 1 || gm > 1024 ||
        (sp != 1 && sp != 2 && sp != 4))
      return fail(TG_ERR_INVALID_ARG, "malformed tuning entry in " + std::string(path));
    const int b = tune_bucket(mm);
    kern[b] = single ? TUNE_SINGLE : TUNE_PAIR;
    grp[b] = (int)gm;
    spl[b] = (int)sp;
    ++entries;
    pos = close;
  }
  if (entries == 0 && j.find("\"min_markers\"") != std::string::npos)
    return fail(TG_ERR_INVALID_ARG, "malformed tuning file " + std::string(path));
  std::memcpy(c->tune_kernel, kern, sizeof(kern));
  std::memcpy(c->tune_group, grp, sizeof(grp));
  std::memcpy(c->tune_split, spl, sizeof(spl));
  return TG_OK;
}

tg_status tg_tuning(const tg_ctx* c, int64_t M, int32_t* kernel, int32_t* group) {
  TG_ARG(c && M > 0, "bad arguments");
  const int b = tune_bucket(M);
  if (kernel) *kernel = c->tune_kernel[b] == TUNE_SINGLE ? 1 : 2;
  if (group) *group = c->tune_group[b] > 0 ? c->tune_group[b] : kGroupDefault;
  return TG_OK;
}

}  // extern "C"
