"""Helpers shared by the GPU parity tests: run the library through its C ABI, run the
oracle on the same inputs, and compare within the stated tolerances.

Tolerances (split BF16 and FP32 forms), derived from the arithmetic of the two forms:
  |d r|           <= r_tol(df) = 5e-7 + 4e-5 / sqrt(df)
                     (accumulation bias plus the random error of the bf16 hi+lo panel,
                      sigma = 2^-17/sqrt(3) * |a|/|a_res| / sqrt(N), taken at 5 sigma)
  |d -log10 p|    <= max(1e-3, 1e-5 * (-log10 p))
  |d beta|        <= 1e-4 * max(|beta|, se)
  |d se|          <= 1e-4 * se
  |d t|           <= r_tol * sqrt(df) / (1 - r^2)^1.5 + 1e-6 |t|
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

import oracle
import paper_2604_21095_gb300 as tg

def r_tol(df) -> float:
    return 5e-7 + 4e-5 / math.sqrt(df)


HIT_DTYPE = np.dtype([("marker", "<u4"), ("pheno", "<u4"), ("beta", "<f4"), ("se", "<f4"),
                      ("t", "<f4"), ("mlog10p", "<f4")])


def enc_id(encoding: str) -> int:
    return tg.TG_ENC_2BIT if encoding == "2bit" else tg.TG_ENC_U8_DOSAGE


def prec_id(precision: str) -> int:
    return {"split": tg.TG_PREC_SPLIT_BF16, "fp32": tg.TG_PREC_FP32,
            "fp4": tg.TG_PREC_FP4_PIECES}[precision]


def run_scan(ctx, panel, G, N, P, encoding, precision, full=True, hit_mlog10p=0.0,
             hit_capacity=1 << 16, missing=None, marker_offset=0, stream=None,
             mode=tg.TG_MODE_PROJECTED):
    """One tg_scan_block call; returns a dict of numpy arrays."""
    dev = G.device
    M = G.shape[0]
    o = {}
    if full:
        for k in ("beta", "se", "t", "mlog10p"):
            o[k] = torch.full((M, P), float("nan"), dtype=torch.float32, device=dev)
    hits = torch.zeros(hit_capacity * HIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
    best = torch.zeros(P, dtype=torch.int64, device=dev)
    norm2 = torch.full((M,), float("nan"), dtype=torch.float64, device=dev)
    nobs = torch.zeros(M, dtype=torch.int32, device=dev)
    mean = torch.zeros(M, dtype=torch.float64, device=dev)
    out = tg.make_outputs(beta=o.get("beta"), se=o.get("se"), t=o.get("t"),
                          mlog10p=o.get("mlog10p"), ldo=P, hits=hits, n_hits=n_hits, best=best,
                          marker_norm2=norm2, marker_nobs=nobs, marker_mean=mean)
    opts = tg.tg_scan_opts(prec_id(precision), 1 if full else 0, float(hit_mlog10p), mode)
    tg.tg_scan_block(ctx, panel, G, N, M, enc_id(encoding), opts, out, marker_offset=marker_offset,
                     missing=missing, stream=stream)
    status = tg.tg_status_poll(ctx, stream)
    torch.cuda.synchronize()
    nh = int(n_hits.item())
    res = {k: v.cpu().numpy() for k, v in o.items()}
    res["status"] = status
    res["n_hits"] = nh
    res["hits"] = np.frombuffer(hits.cpu().numpy().tobytes(), dtype=HIT_DTYPE)[: min(nh, hit_capacity)]
    b = best.cpu().numpy().view(np.uint64)
    res["best_key"] = b
    res["best_marker"] = np.where(b == 0, -1, (0xFFFFFFFF - (b & 0xFFFFFFFF)).astype(np.int64))
    res["best_absr"] = np.frombuffer(((b >> 32).astype(np.uint32)).tobytes(), dtype=np.float32)
    res["norm2"] = norm2.cpu().numpy()
    res["nobs"] = nobs.cpu().numpy()
    res["mean"] = mean.cpu().numpy()
    return res


def oracle_panel(Yt: torch.Tensor, cov_t, samples=None):
    Y = Yt.cpu().numpy().T.astype(np.float64)
    C = None if cov_t is None or cov_t.shape[0] == 0 else cov_t.cpu().numpy().T
    return oracle.prepare_panel(Y, C, samples)


def sample_words(rows: np.ndarray) -> torch.Tensor:
    """bool [N] -> int32 words [ceil(N/32)], bit i%32 of word i/32 = rows[i]."""
    N = rows.shape[0]
    w = np.zeros((N + 31) // 32, dtype=np.uint32)
    for i in np.nonzero(rows)[0]:
        w[i // 32] |= np.uint32(1) << np.uint32(i % 32)
    return torch.from_numpy(w.view(np.int32).copy())


def compare_full(res, ref, label="", rtol=None):
    """Element-wise comparison of FULL outputs against the projected oracle; returns max errors."""
    df = ref["df"]
    rtol = r_tol(df) if rtol is None else rtol
    r = ref["r"]
    ok = np.isfinite(r)
    assert np.array_equal(np.isfinite(res["t"]), ok), f"{label}: NaN pattern differs"
    rb = res["t"] / np.sqrt(df + res["t"].astype(np.float64) ** 2)  # r from t
    err = {}
    dr = np.abs(rb - r)[ok]
    err["r"] = float(dr.max()) if dr.size else 0.0
    mlp_o = ref["mlog10p"][ok]
    dm = np.abs(res["mlog10p"][ok] - mlp_o)
    err["mlog10p"] = float(dm.max()) if dm.size else 0.0
    assert np.all(dm <= np.maximum(1e-3, 1e-5 * mlp_o)), f"{label}: -log10 p max err {err['mlog10p']}"
    se_o = ref["se"][ok]
    db = np.abs(res["beta"][ok] - ref["beta"][ok])
    err["beta_rel_se"] = float((db / np.maximum(np.abs(ref["beta"][ok]), se_o)).max()) if db.size else 0.0
    assert np.all(db <= 1e-4 * np.maximum(np.abs(ref["beta"][ok]), se_o)), f"{label}: beta err {err['beta_rel_se']}"
    ds = np.abs(res["se"][ok] - se_o)
    err["se_rel"] = float((ds / se_o).max()) if ds.size else 0.0
    assert np.all(ds <= 1e-4 * se_o), f"{label}: se err {err['se_rel']}"
    dt = np.abs(res["t"][ok] - ref["t"][ok])
    rr = np.abs(r[ok])
    bound = rtol * math.sqrt(df) / np.maximum((1 - rr * rr), 1e-12) ** 1.5 + 1e-6 * np.abs(ref["t"][ok])
    err["t"] = float(dt.max()) if dt.size else 0.0
    assert np.all(dt <= bound), f"{label}: t err {err['t']}"
    assert err["r"] <= rtol * 1.01 + 1e-7, f"{label}: r err {err['r']}"
    return err


def compare_hits(res, ref, thr, marker_offset=0, tol_band=None):
    """GPU hits vs oracle hits: equal sets except pairs within the -log10 p tolerance of the
    threshold; every GPU hit's statistics within tolerance of the oracle's."""
    mlp = ref["mlog10p"]
    want = {tuple(x) for x in oracle.hits(mlp, thr, marker_offset).tolist()}
    got = {(int(h["marker"]), int(h["pheno"])) for h in res["hits"]}
    assert res["n_hits"] == len(res["hits"]), "hit buffer overflowed in a parity test"
    for m, p in want ^ got:
        v = mlp[m - marker_offset, p]
        band = max(1e-3, 1e-5 * abs(v)) if tol_band is None else tol_band
        assert abs(v - thr) <= band, f"hit ({m},{p}) oracle -log10p {v} not near threshold {thr}"
    for h in res["hits"]:
        j, p = int(h["marker"]) - marker_offset, int(h["pheno"])
        mo = mlp[j, p]
        assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (j, p, h["mlog10p"], mo)
        assert abs(h["beta"] - ref["beta"][j, p]) <= 1e-4 * max(abs(ref["beta"][j, p]), ref["se"][j, p])
    return len(want), len(got)


def compare_best(res, ref, rtol=None, marker_offset=0, rel=0.0):
    """Per phenotype the GPU's best marker is a valid argmax of |r| within the r tolerance.

    The best key holds |r| from the FP32 product; `rel` adds a tolerance proportional to |r| for
    cases with |r| close to 1, where the tensor-core accumulation's rounding of a sum of terms of
    one sign is relative to |r| rather than to the terms (returned: the largest deviation)."""
    rtol = r_tol(ref["df"]) if rtol is None else rtol
    absr = np.nan_to_num(np.abs(ref["r"]), nan=-1.0)  # untestable markers rank below all
    worst = 0.0
    for p in range(absr.shape[1]):
        col = absr[:, p]
        if col.max() < 0:
            assert res["best_marker"][p] == -1
            continue
        j = res["best_marker"][p] - marker_offset
        assert 0 <= j < col.size
        tol = rtol * 2 + 1e-7 + rel * col.max()
        assert col[j] >= col.max() - tol, (p, j, col[j], col.max())
        dev = abs(float(res["best_absr"][p]) - col[j])
        worst = max(worst, dev)
        assert dev <= tol, (p, j, float(res["best_absr"][p]), col[j], dev)
    return worst
