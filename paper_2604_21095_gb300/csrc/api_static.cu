// tg_scan_block_static: the block scan for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc or cudaFree at scan time: code that runs inside a
// host application whose device memory is owned by another allocator (a framework's caching
// pool or a fixed memory budget handed out elsewhere), and latency-critical loops where the
// device-wide synchronisation that cudaMalloc/cudaFree can trigger is not acceptable. For
// them this entry point runs the same kernels as tg_scan_block, but every piece of scratch
// memory (the decoded genotype operand, the per-marker statistics, the status word) lives in
// one file-scope __device__ array of kStaticScratchBytes, which each GPU that loads the
// library keeps until the process exits. The caller still passes the panel, the inputs and
// the outputs. Nothing here calls cudaMalloc, cudaFree or any allocating library routine.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

using namespace tg;

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB on every device that loads the library
constexpr int kMaxDevices = 64;
constexpr long long kStaticSpinNs = 4000000000ll;

// The scratch. In host code this name is a host-side stand-in, not a device address: the
// device address comes from cudaGetSymbolAddress, once per device, in set_up().
static __device__ __align__(256) unsigned char g_scan_scratch[kStaticScratchBytes];

struct DeviceState {
  unsigned char* base = nullptr;  // device address of g_scan_scratch on this device
  int sm_count = 0;
  bool ready = false;
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_static() {
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

bool tmap_static(CUtensorMap* m, const void* ptr, int64_t rows, int64_t K, int64_t ld,
                 uint32_t box_rows) {
  auto fn = encode_fn_static();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {32u, box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-device set-up, done by the first call on a device with that device current.
tg_status set_up(int dev, DeviceState** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return fail(TG_ERR_UNSUPPORTED, "device index too large");
  DeviceState& s = g_state[dev];
  if (!s.ready) {
    int major = 0, minor = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) ||
        (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      return cuda_fail(e, "tg_scan_block_static: device attributes");
    if (!(major == 10 && minor == 3)) return fail(TG_ERR_UNSUPPORTED, "needs an sm_103 (GB300) device");
    if (!encode_fn_static()) return fail(TG_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scan_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "tg_scan_block_static: cudaGetSymbolAddress");
    s.base = static_cast<unsigned char*>(p);
    s.sm_count = sms;
    s.ready = true;
  }
  *out = &s;
  return TG_OK;
}

// Carves aligned pieces out of the scratch.
struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

extern "C" tg_status tg_scan_block_static(const tg_panel* p, const uint8_t* G, int64_t ldg,
                                          int32_t encoding, int64_t N, int64_t M,
                                          int64_t marker_offset, const uint32_t* missing,
                                          int64_t ldm, const tg_scan_opts* opts,
                                          const tg_outputs* out, void* stream) {
  if (!p || !opts || !out) return fail(TG_ERR_INVALID_ARG, "null panel, options or outputs");
  if (encoding != TG_ENC_2BIT && encoding != TG_ENC_U8_DOSAGE)
    return fail(TG_ERR_INVALID_ARG, "unknown encoding");
  const int prec = opts->precision;
  if (prec == TG_PREC_FP4_PIECES)
    return fail(TG_ERR_UNSUPPORTED, "the FP4 form is scanned with tg_scan_block, not the static form");
  if (prec != TG_PREC_FP32 && prec != TG_PREC_SPLIT_BF16) return fail(TG_ERR_INVALID_ARG, "unknown precision");
  if ((opts->mode != TG_MODE_PROJECTED && opts->mode != TG_MODE_PAPER) || opts->reserved != 0)
    return fail(TG_ERR_INVALID_ARG, "unknown mode (or tg_scan_opts.reserved != 0)");
  if (p->samples)
    return fail(TG_ERR_UNSUPPORTED, "subset panels are scanned with tg_scan_block, not the static form");
  if (N != p->N) return fail(TG_ERR_INVALID_ARG, "N differs from the panel's sample count");
  if (M < 0 || marker_offset < 0 || marker_offset + M > 0xFFFFFFFFll)
    return fail(TG_ERR_INVALID_ARG, "bad M or marker_offset");
  if (M == 0) return TG_OK;
  if (!G || reinterpret_cast<uintptr_t>(G) % 16) return fail(TG_ERR_INVALID_ARG, "G must be 16-byte aligned");
  const int64_t need = encoding == TG_ENC_2BIT ? (N + 3) / 4 : N;
  if (ldg < need || ldg % 16) return fail(TG_ERR_INVALID_ARG, "ldg must be >= the row length and a multiple of 16");
  if (encoding == TG_ENC_2BIT && missing) return fail(TG_ERR_INVALID_ARG, "missing must be NULL for 2-bit calls");
  if (missing && ldm < (N + 31) / 32) return fail(TG_ERR_INVALID_ARG, "ldm too small");
  if (opts->full_output && (out->ldo < p->P || !(out->beta || out->se || out->t || out->mlog10p)))
    return fail(TG_ERR_INVALID_ARG, "full_output needs ldo >= P and an output array");
  const bool want_hits = opts->hit_mlog10p > 0.0;
  if (want_hits && (!out->n_hits || out->hit_capacity < 0 || (!out->hits && out->hit_capacity > 0)))
    return fail(TG_ERR_INVALID_ARG, "hit collection needs hits, hit_capacity and n_hits");

  // size check before anything is touched
  const bool split = prec == TG_PREC_SPLIT_BF16;
  const int64_t rows = round_up(M, MT);
  const size_t elem = prec == TG_PREC_FP32 ? 4 : 2;
  Carver probe{nullptr};
  probe.take<uint32_t>(4);
  probe.take<unsigned long long>(1);
  probe.take<float>((size_t)rows);
  probe.take<int32_t>((size_t)rows);
  probe.take<double>((size_t)rows);
  probe.take<double>((size_t)rows);
  probe.take<float>((size_t)rows * QCOLS);
  probe.take<double>((size_t)rows);
  probe.take<float>((size_t)rows);
  probe.take<double>((size_t)rows);
  probe.take<int>((size_t)rows);
  probe.take<unsigned char>((size_t)rows * p->Npad * elem);
  if (probe.used > kStaticScratchBytes) {
    const size_t per = (size_t)p->Npad * elem + 4 * QCOLS + 64;
    return fail(TG_ERR_UNSUPPORTED,
                "block too large for the 64 MiB static scratch: at most about " +
                    std::to_string(kStaticScratchBytes / per) + " markers at N = " +
                    std::to_string(N) + " in this precision");
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != p->device) return fail(TG_ERR_INVALID_ARG, "the panel lives on another device");
  DeviceState* ds = nullptr;
  tg_status s = set_up(dev, &ds);
  if (s != TG_OK) return s;

  Carver cv{ds->base};
  uint32_t* status = cv.take<uint32_t>(4);  // [0] status word, [1] count of re-projected markers
  unsigned long long* hit_start = cv.take<unsigned long long>(1);
  float* shift = cv.take<float>((size_t)rows);
  int32_t* nobs = cv.take<int32_t>((size_t)rows);
  double* mean = cv.take<double>((size_t)rows);
  double* gc2 = cv.take<double>((size_t)rows);
  float* qg = cv.take<float>((size_t)rows * QCOLS);
  double* gres2 = cv.take<double>((size_t)rows);
  float* rinv = cv.take<float>((size_t)rows);
  double* rinv64 = cv.take<double>((size_t)rows);
  int* refine_list = cv.take<int>((size_t)rows);
  void* Ahi = cv.take<unsigned char>((size_t)rows * p->Npad * elem);

  cudaStream_t st = (cudaStream_t)stream;
  const double kappa64 = encoding == TG_ENC_U8_DOSAGE ? 2.0 / 255.0 : 1.0;
  const float kappa = (float)kappa64;
#define TGS_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)
  // every call shares the scratch and it keeps the last call's contents: clear what must start at 0
  TGS_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
  TGS_CUDA(launch_decode(G, ldg, encoding, N, M, missing, ldm, prec, Ahi,
                         split ? shift : nullptr, nullptr, p->Npad, nobs, nullptr, nullptr, mean,
                         gc2, st));
  CUtensorMap tA;
  if (split && !tmap_static(&tA, Ahi, M, p->Npad, p->Npad, MT))
    return fail(TG_ERR_CUDA, "cuTensorMapEncodeTiled failed for the genotype operand");
  const int64_t nq = opts->mode == TG_MODE_PAPER ? 0 : p->q - 1;  // the paper's form: no projection
  // a small panel: the projection and the panel's products in one pass (raw, into qg)
  const bool joint = split && nq > 0 && p->joint_cols == QCOLS;  // the scratch holds 64 columns
  if (nq > 0) {
    if (!split) {
      TGS_CUDA(launch_project(reinterpret_cast<const float*>(Ahi), p->Npad, M, p->Npad, p->QB, nq,
                              qg, st));
    } else {
      EpiParams pp{};
      pp.M = (int)M;
      pp.P = (int)(joint ? nq + p->P : nq);
      pp.status = status;
      pp.row_shift = shift;
      pp.col_cs = joint ? p->qycs : p->qcs;
      pp.raw_out = qg;
      pp.raw_cols = pp.P;
      pp.raw_ld = QCOLS;
      TGS_CUDA(launch_tc_scan(&tA, joint ? &p->tmQYhi : &p->tmQhi, joint ? &p->tmQYlo : &p->tmQlo,
                              p->Npad, pp, ds->sm_count, kStaticSpinNs, st));
    }
  }
  const MarkerRefine rf{G, ldg, encoding, N, missing, ldm, mean, p->Q, (int)p->q, refine_list,
                        status + 1};
  TGS_CUDA(launch_marker_norm(M, nobs, gc2, qg, QCOLS, nq, kappa64, gres2, out->marker_norm2, rinv, rinv64,
                              &rf, st));
  if (out->marker_nobs)
    TGS_CUDA(cudaMemcpyAsync(out->marker_nobs, nobs, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
  if (out->marker_mean)
    TGS_CUDA(cudaMemcpyAsync(out->marker_mean, mean, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
  EpiParams ep{};
  ep.M = (int)M;
  ep.P = (int)p->P;
  ep.marker_offset = marker_offset;
  mode_df(p, opts->mode, &ep.df, &ep.lnB);
  ep.df_f = (float)ep.df;
  ep.kappa = kappa;
  ep.kappa64 = kappa64;
  ep.do_hits = want_hits ? 1 : 0;
  ep.r2_thr = want_hits ? (float)host_r2_threshold(opts->hit_mlog10p, ep.df, ep.lnB) : 2.0f;
  ep.do_full = opts->full_output ? 1 : 0;
  ep.do_best = out->best != nullptr;
  ep.row_inv = rinv;
  ep.row_inv64 = rinv64;
  ep.exact = ExactArgs{G, ldg, encoding, (int)N, missing, ldm, mean, p->Yres, p->N};
  ep.col_s = p->col_s;
  ep.col_s64 = p->s;
  ep.col_rmul = p->col_rmul;
  ep.row_shift = split ? shift : nullptr;
  ep.col_cs = p->col_cs;
  ep.beta = out->beta;
  ep.se = out->se;
  ep.t = out->t;
  ep.mlp = out->mlog10p;
  ep.rstore = out->t ? out->t : out->mlog10p ? out->mlog10p : out->beta ? out->beta : out->se;
  ep.ldo = out->ldo;
  ep.hits = out->hits;
  ep.hit_cap = out->hit_capacity;
  ep.n_hits = out->n_hits;
  ep.best = out->best;
  ep.status = status;
  if (ep.do_hits)
    TGS_CUDA(cudaMemcpyAsync(hit_start, ep.n_hits, sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, st));
  if (!split) {
    TGS_CUDA(launch_sgemm_scan(reinterpret_cast<const float*>(Ahi), p->Npad, p->B32, p->Npad,
                               p->Npad, ep, st));
  } else if (joint) {  // the products came with the projection
    TGS_CUDA(launch_raw_stats(qg + nq, QCOLS, ep, st));
  } else {
    const bool narrow = p->P <= 64;  // a small panel: 64-column tiles, bound by HBM
    TGS_CUDA(launch_tc_scan(&tA, narrow ? &p->tmBhi64 : &p->tmBhi, narrow ? &p->tmBlo64 : &p->tmBlo,
                            p->Npad, ep, ds->sm_count, kStaticSpinNs, st, 16, nullptr, 0, narrow));
  }
  if (ep.do_hits) TGS_CUDA(launch_hit_stats(ep, hit_start, st));
  if (ep.do_full) TGS_CUDA(launch_full_stats(ep, st));
  // synchronous: the device status of this call is returned
  uint32_t word = 0;
  TGS_CUDA(cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st));
  TGS_CUDA(cudaStreamSynchronize(st));
#undef TGS_CUDA
  if (word & ST_TIMEOUT) return fail(TG_ERR_TIMEOUT, "a bounded device wait ran out");
  if (word & ST_CAPACITY) return fail(TG_ERR_CAPACITY, "more hits than hit_capacity");
  return TG_OK;
}
