"""ctypes binding of libtg.so: the C entry points under the same names, argument marshalling only.

Tensor arguments are torch tensors on the context's CUDA device (or None where the C call
accepts NULL); their data pointers and leading dimensions are passed through unchanged.
Every computation runs in the library's CUDA kernels. A failed call raises TgError with
the library's status and message. The library must have been built (see build.py); the
binding never falls back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TG_OK, TG_ERR_INVALID_ARG, TG_ERR_CUDA, TG_ERR_OOM, TG_ERR_NONFINITE, TG_ERR_RANK, \
    TG_ERR_CAPACITY, TG_ERR_TIMEOUT, TG_ERR_UNSUPPORTED = range(9)
TG_PREC_FP32, TG_PREC_SPLIT_BF16, TG_PREC_FP4_PIECES = 0, 1, 2
TG_ENC_2BIT, TG_ENC_U8_DOSAGE = 0, 1
TG_MODE_PROJECTED, TG_MODE_PAPER = 0, 1
TG_N_STAGES = 6
STAGES = ("decode", "project", "norm", "scan", "h2d", "stats")


class TgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tg status {status}: {msg}")
        self.status = status


class tg_scan_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("full_output", C.c_int32), ("hit_mlog10p", C.c_double),
                ("mode", C.c_int32), ("reserved", C.c_int32)]


class tg_hit(C.Structure):
    _fields_ = [("marker", C.c_uint32), ("pheno", C.c_uint32), ("beta", C.c_float),
                ("se", C.c_float), ("t", C.c_float), ("mlog10p", C.c_float)]


class tg_outputs(C.Structure):
    _fields_ = [("beta", C.c_void_p), ("se", C.c_void_p), ("t", C.c_void_p),
                ("mlog10p", C.c_void_p), ("ldo", C.c_int64), ("hits", C.c_void_p),
                ("hit_capacity", C.c_int64), ("n_hits", C.c_void_p), ("best", C.c_void_p),
                ("marker_norm2", C.c_void_p), ("marker_nobs", C.c_void_p),
                ("marker_mean", C.c_void_p)]


_VP, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_SIGS = {
    "tg_version": (C.c_char_p, []),
    "tg_abi_version": (C.c_int, []),
    "tg_last_error": (C.c_char_p, []),
    "tg_status_string": (C.c_char_p, [C.c_int]),
    "tg_create": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "tg_destroy": (C.c_int, [_VP]),
    "tg_prepare_panel": (C.c_int, [_VP, _VP, _I64, _I64, _I64, _VP, _I64, _I64, C.POINTER(_VP), _VP]),
    "tg_panel_info": (C.c_int, [_VP, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    "tg_panel_Q": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_I64), C.POINTER(_I64)]),
    "tg_panel_Yres": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_I64), C.POINTER(_VP)]),
    "tg_panel_free": (C.c_int, [_VP]),
    "tg_decode_block": (C.c_int, [_VP, _VP, _I64, _I32, _I64, _I64, _VP, _I64, _I32, _VP, _VP,
                                  _I64, _VP, _VP, _VP, _VP, _VP]),
    "tg_scan_block": (C.c_int, [_VP, _VP, _VP, _I64, _I32, _I64, _I64, _I64, _VP, _I64,
                                C.POINTER(tg_scan_opts), C.POINTER(tg_outputs), _VP]),
    "tg_scan_block_static": (C.c_int, [_VP, _VP, _I64, _I32, _I64, _I64, _I64, _VP, _I64,
                                       C.POINTER(tg_scan_opts), C.POINTER(tg_outputs), _VP]),
    "tg_scan_host": (C.c_int, [_VP, _VP, _VP, _I64, _I32, _I64, _I64, _I64, _I64,
                               C.POINTER(tg_scan_opts), _VP, _I64, C.POINTER(_I64), _VP, _VP]),
    "tg_panel_concat": (C.c_int, [_VP, C.POINTER(_VP), C.c_int, C.POINTER(_VP), _VP]),
    "tg_tuning_save": (C.c_int, [_VP, C.c_char_p]),
    "tg_tuning_load": (C.c_int, [_VP, C.c_char_p]),
    "tg_set_tuning_split": (C.c_int, [_VP, _I64, _I32]),
    "tg_tuning_split": (C.c_int, [_VP, _I64, C.POINTER(_I32)]),
    "tg_set_host_ramp": (C.c_int, [_VP, C.c_double]),
    "tg_set_host_buffers": (C.c_int, [_VP, C.c_int]),
    "tg_host_ramp": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tg_host_block_sizes": (C.c_int, [_I64, _I64, C.c_double, C.POINTER(_I64), _I64,
                                      C.POINTER(_I64)]),
    "tg_scan_graph_create": (C.c_int, [_VP, _VP, C.c_int, C.POINTER(_VP), C.POINTER(_I64),
                                       C.POINTER(_I64), C.POINTER(_VP), _I64, _I64, _I32, _I64,
                                       C.POINTER(tg_scan_opts), C.POINTER(tg_outputs),
                                       C.POINTER(_VP)]),
    "tg_scan_graph_create_host": (C.c_int, [_VP, _VP, C.c_int, C.POINTER(_VP), C.POINTER(_I64),
                                            C.POINTER(_I64), _I64, _I32, _I64,
                                            C.POINTER(tg_scan_opts), C.POINTER(tg_outputs),
                                            C.POINTER(_VP)]),
    "tg_scan_graph_launch": (C.c_int, [_VP, _VP]),
    "tg_scan_graph_free": (C.c_int, [_VP]),
    "tg_autotune": (C.c_int, [_VP, _VP, _I32, _I64, _VP]),
    "tg_tuning": (C.c_int, [_VP, _I64, C.POINTER(_I32), C.POINTER(_I32)]),
    "tg_set_tuning": (C.c_int, [_VP, _I64, _I32, _I32]),
    "tg_status_poll": (C.c_int, [_VP, _VP]),
    "tg_set_fused_decode": (C.c_int, [_VP, C.c_int]),
    "tg_prepare_panel_subset": (C.c_int, [_VP, _VP, _I64, _I64, _I64, _VP, _I64, _I64, _VP,
                                          C.POINTER(_VP), _VP]),
    "tg_panel_samples": (C.c_int, [_VP, C.POINTER(_I64), C.POINTER(_VP)]),
    "tg_phenotype_masks": (C.c_int, [_VP, _VP, _I64, _I64, _I64, _VP, _I64, _VP]),
    "tg_set_profiling": (C.c_int, [_VP, C.c_int]),
    "tg_stage_times": (C.c_int, [_VP, C.POINTER(_D), C.POINTER(_I64), C.c_int]),
    "tg_bounded_wait_test": (C.c_int, [_VP, _VP, _I64, _VP]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libtg.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libtg.so is not built: run paper_2604_21095_gb300.build.build() "
                               "(or __graft_entry__.build()) first")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols():
    return list(_SIGS)


def _check(status: int):
    if status != TG_OK:
        raise TgError(status, load().tg_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ld(t):
    """Leading dimension of a tensor stored as [rows][ld] (row stride in elements)."""
    return t.stride(0) if t.dim() == 2 else t.numel()


# ---------------------------------------------------------------- entry points

def tg_version() -> str:
    return load().tg_version().decode()


def tg_abi_version() -> int:
    return load().tg_abi_version()


def tg_last_error() -> str:
    return load().tg_last_error().decode()


def tg_status_string(s: int) -> str:
    return load().tg_status_string(s).decode()


def tg_create(device: int = 0):
    h = _VP()
    _check(load().tg_create(C.byref(h), device))
    return h


def tg_destroy(ctx):
    _check(load().tg_destroy(ctx))


def tg_prepare_panel(ctx, Y, N, P, C_cov=None, stream=None):
    """Y: float32 tensor [P][ldy] (column-major N x P); C_cov: float64 [n_cov][ldc] or None."""
    out = _VP()
    n_cov = 0 if C_cov is None else C_cov.shape[0]
    ldc = N if C_cov is None else _ld(C_cov)
    _check(load().tg_prepare_panel(ctx, _ptr(Y), _ld(Y), N, P, _ptr(C_cov), ldc, n_cov,
                                   C.byref(out), _stream(stream)))
    return out


def tg_panel_info(panel):
    v = [_I64() for _ in range(4)]
    _check(load().tg_panel_info(panel, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


class _Borrowed:
    """__cuda_array_interface__ view of a device buffer owned by the library."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _view(ptr, shape, typestr):
    import torch
    return torch.as_tensor(_Borrowed(ptr, shape, typestr), device="cuda")


def tg_panel_Q(panel):
    """Borrowed FP64 Q as a tensor [q][N] (column-major N x q)."""
    p, ld, q = _VP(), _I64(), _I64()
    _check(load().tg_panel_Q(panel, C.byref(p), C.byref(ld), C.byref(q)))
    return _view(p.value, (q.value, ld.value), "<f8")


def tg_panel_Yres(panel):
    """Borrowed FP64 (Y_res [P][N], s [P])."""
    N, P, _, _ = tg_panel_info(panel)
    p, ld, s = _VP(), _I64(), _VP()
    _check(load().tg_panel_Yres(panel, C.byref(p), C.byref(ld), C.byref(s)))
    return _view(p.value, (P, ld.value), "<f8"), _view(s.value, (P,), "<f8")


def tg_panel_free(panel):
    _check(load().tg_panel_free(panel))


def tg_decode_block(ctx, G, N, M, encoding, precision, A, shift=None, missing=None,
                    n_obs=None, S=None, S2=None, mean=None, stream=None):
    ldm = _ld(missing) if missing is not None else 0
    _check(load().tg_decode_block(ctx, _ptr(G), _ld(G), encoding, N, M, _ptr(missing), ldm,
                                  precision, _ptr(A), _ptr(shift), _ld(A), _ptr(n_obs),
                                  _ptr(S), _ptr(S2), _ptr(mean), _stream(stream)))


def make_outputs(beta=None, se=None, t=None, mlog10p=None, ldo=0, hits=None, n_hits=None,
                 best=None, marker_norm2=None, marker_nobs=None, marker_mean=None) -> tg_outputs:
    """hits: uint8 tensor of capacity*24 bytes (tg_hit records) or None."""
    cap = 0 if hits is None else hits.numel() * hits.element_size() // C.sizeof(tg_hit)
    return tg_outputs(_ptr(beta), _ptr(se), _ptr(t), _ptr(mlog10p), ldo, _ptr(hits), cap,
                      _ptr(n_hits), _ptr(best), _ptr(marker_norm2), _ptr(marker_nobs),
                      _ptr(marker_mean))


def tg_scan_block(ctx, panel, G, N, M, encoding, opts: tg_scan_opts, out: tg_outputs,
                  marker_offset=0, missing=None, stream=None):
    ldm = _ld(missing) if missing is not None else 0
    _check(load().tg_scan_block(ctx, panel, _ptr(G), _ld(G), encoding, N, M, marker_offset,
                                _ptr(missing), ldm, C.byref(opts), C.byref(out), _stream(stream)))


def tg_scan_block_static(panel, G, N, M, encoding, opts: tg_scan_opts, out: tg_outputs,
                         marker_offset=0, missing=None, stream=None):
    """tg_scan_block without a context and without any device allocation (static scratch).
    Synchronous; raises TgError on failure (including TG_ERR_CAPACITY / TG_ERR_TIMEOUT)."""
    ldm = _ld(missing) if missing is not None else 0
    _check(load().tg_scan_block_static(panel, _ptr(G), _ld(G), encoding, N, M, marker_offset,
                                       _ptr(missing), ldm, C.byref(opts), C.byref(out),
                                       _stream(stream)))


def tg_scan_host(ctx, panel, G_host, N, M, encoding, block_markers, opts: tg_scan_opts,
                 hits_host, best_host=None, marker_offset=0, stream=None):
    """G_host: uint8 CPU tensor [M][ldg] (pinned for overlap); hits_host: uint8 CPU tensor of
    capacity*24 bytes; best_host: uint64-sized CPU tensor [P] or None. Returns the hit count."""
    n = _I64()
    cap = hits_host.numel() * hits_host.element_size() // C.sizeof(tg_hit)
    st = load().tg_scan_host(ctx, panel, _ptr(G_host), _ld(G_host), encoding, N, M, block_markers,
                             marker_offset, C.byref(opts), _ptr(hits_host), cap, C.byref(n),
                             _ptr(best_host), _stream(stream))
    if st == TG_ERR_CAPACITY:
        return n.value
    _check(st)
    return n.value


def tg_panel_concat(ctx, panels, stream=None):
    """One panel whose columns are the given panels' columns, in order."""
    arr = (_VP * len(panels))(*[p.value if isinstance(p, _VP) else p for p in panels])
    out = _VP()
    _check(load().tg_panel_concat(ctx, arr, len(panels), C.byref(out), _stream(stream)))
    return out


def tg_scan_graph_create(ctx, panel, blocks, N, encoding, opts: tg_scan_opts, out: tg_outputs,
                         marker_offsets, missing=None):
    """blocks: list of uint8 device tensors [M_b][ldg] (same ldg); returns a graph handle."""
    n = len(blocks)
    G = (_VP * n)(*[b.data_ptr() for b in blocks])
    M = (_I64 * n)(*[b.shape[0] for b in blocks])
    off = (_I64 * n)(*marker_offsets)
    miss = None
    ldm = 0
    if missing is not None:
        miss = (_VP * n)(*[_ptr(m) for m in missing])
        ldm = next(_ld(m) for m in missing if m is not None)
    g = _VP()
    _check(load().tg_scan_graph_create(ctx, panel, n, G, M, off, miss, _ld(blocks[0]), ldm,
                                       encoding, N, C.byref(opts), C.byref(out), C.byref(g)))
    return g


def tg_scan_graph_create_host(ctx, panel, blocks_host, N, encoding, opts: tg_scan_opts,
                              out: tg_outputs, marker_offsets):
    """blocks_host: list of uint8 CPU tensors [M_b][ldg] in page-locked memory (same ldg); the
    graph copies them to the device at every replay. Returns a graph handle."""
    n = len(blocks_host)
    G = (_VP * n)(*[b.data_ptr() for b in blocks_host])
    M = (_I64 * n)(*[b.shape[0] for b in blocks_host])
    off = (_I64 * n)(*marker_offsets)
    g = _VP()
    _check(load().tg_scan_graph_create_host(ctx, panel, n, G, M, off, _ld(blocks_host[0]),
                                            encoding, N, C.byref(opts), C.byref(out), C.byref(g)))
    return g


def tg_scan_graph_launch(graph, stream=None):
    _check(load().tg_scan_graph_launch(graph, _stream(stream)))


def tg_scan_graph_free(graph):
    _check(load().tg_scan_graph_free(graph))


def tg_autotune(ctx, panel, encoding, M, stream=None):
    _check(load().tg_autotune(ctx, panel, encoding, M, _stream(stream)))


def tg_tuning(ctx, M):
    k, g = _I32(), _I32()
    _check(load().tg_tuning(ctx, M, C.byref(k), C.byref(g)))
    return {"kernel": "pair" if k.value == 2 else "single", "group_m": g.value}


def tg_set_tuning(ctx, M, kernel: str, group_m: int):
    _check(load().tg_set_tuning(ctx, M, 2 if kernel == "pair" else 1, group_m))


def tg_set_tuning_split(ctx, M, splits: int):
    _check(load().tg_set_tuning_split(ctx, M, splits))


def tg_tuning_split(ctx, M) -> int:
    v = _I32()
    _check(load().tg_tuning_split(ctx, M, C.byref(v)))
    return v.value


def tg_set_host_ramp(ctx, factor: float = 0.0):
    _check(load().tg_set_host_ramp(ctx, float(factor)))


def tg_set_host_buffers(ctx, n_buffers: int = 3):
    _check(load().tg_set_host_buffers(ctx, int(n_buffers)))


def tg_host_ramp(ctx):
    """(factor the next tg_scan_host call uses, last measured scan / copy ratio)."""
    f, r = C.c_double(), C.c_double()
    _check(load().tg_host_ramp(ctx, C.byref(f), C.byref(r)))
    return f.value, r.value


def tg_host_block_sizes(M, block_markers, factor=2.0):
    """The block sizes tg_scan_host streams M markers in (host only)."""
    n = _I64()
    _check(load().tg_host_block_sizes(M, block_markers, float(factor), None, 0, C.byref(n)))
    buf = (_I64 * max(1, n.value))()
    _check(load().tg_host_block_sizes(M, block_markers, float(factor), buf, n.value, C.byref(n)))
    return list(buf[:n.value])


def tg_tuning_save(ctx, path: str):
    _check(load().tg_tuning_save(ctx, os.fsencode(path)))


def tg_tuning_load(ctx, path: str):
    _check(load().tg_tuning_load(ctx, os.fsencode(path)))


def tg_status_poll(ctx, stream=None) -> int:
    """Synchronise and return the latched device status (0 = ok); does not raise."""
    return load().tg_status_poll(ctx, _stream(stream))


def tg_prepare_panel_subset(ctx, Y, N, P, C_cov, samples, stream=None):
    """As tg_prepare_panel, for phenotypes observed on the samples whose bits are set in
    `samples` (int32/uint32 device words [ceil(N/32)])."""
    out = _VP()
    n_cov = 0 if C_cov is None else C_cov.shape[0]
    ldc = N if C_cov is None else _ld(C_cov)
    _check(load().tg_prepare_panel_subset(ctx, _ptr(Y), _ld(Y), N, P, _ptr(C_cov), ldc, n_cov,
                                          _ptr(samples), C.byref(out), _stream(stream)))
    return out


def tg_panel_samples(panel):
    n = _I64()
    m = _VP()
    _check(load().tg_panel_samples(panel, C.byref(n), C.byref(m)))
    return n.value, m.value


def tg_phenotype_masks(ctx, Yt, N, P, masks, stream=None):
    _check(load().tg_phenotype_masks(ctx, _ptr(Yt), _ld(Yt), N, P, _ptr(masks), _ld(masks),
                                     _stream(stream)))


TG_FUSED_OFF, TG_FUSED_ALL, TG_FUSED_SMALL_PANELS = 0, 1, 2


def tg_set_fused_decode(ctx, enable):
    """True / TG_FUSED_ALL: every kernel that can decode in its producer does; False /
    TG_FUSED_OFF: none (the decoded operand always); TG_FUSED_SMALL_PANELS: the default, only the
    joint projection pass of panels with P + q - 1 <= 128."""
    setting = int(enable) if not isinstance(enable, bool) else (TG_FUSED_ALL if enable else TG_FUSED_OFF)
    _check(load().tg_set_fused_decode(ctx, setting))


def tg_set_profiling(ctx, enable: bool):
    _check(load().tg_set_profiling(ctx, 1 if enable else 0))


def tg_stage_times(ctx, reset=False):
    ms = (_D * TG_N_STAGES)()
    n = (_I64 * TG_N_STAGES)()
    _check(load().tg_stage_times(ctx, ms, n, 1 if reset else 0))
    return {STAGES[i]: (ms[i], n[i]) for i in range(TG_N_STAGES)}


def tg_bounded_wait_test(ctx, flag, limit_ns: int, stream=None) -> int:
    """Returns the status (TG_OK when the flag was seen, TG_ERR_TIMEOUT when the limit ran out)."""
    return load().tg_bounded_wait_test(ctx, _ptr(flag), limit_ns, _stream(stream))


def hits_to_numpy(hits_bytes, n):
    """Decode n tg_hit records from a uint8 tensor (device or host) into a numpy structured array."""
    import numpy as np
    dt = np.dtype([("marker", "<u4"), ("pheno", "<u4"), ("beta", "<f4"), ("se", "<f4"),
                   ("t", "<f4"), ("mlog10p", "<f4")])
    raw = hits_bytes[: n * dt.itemsize].cpu().numpy().tobytes()
    return np.frombuffer(raw, dtype=dt, count=n)
