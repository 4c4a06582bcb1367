"""GPU parity at the method's own edge: correlations close to 1 at large df (Section 2.2, the
conversion of r through Eq. 3 to a P value).

At df ~ 23,000 the slope of -log10 p in r, df |r| / ((1 - r^2) ln 10), is about 5e7 at
|r| = 0.9999, so the FP32 product's rounding (~1e-7 in r) would move -log10 p by several units.
Hits and FULL elements with 1 - r^2 < 0.05 therefore take an FP64 product, an FP64 r and the
FP64 continued fraction. These tests plant phenotypes y = b g_j + covariates + noise with
|r| in {0.99, 0.999, 0.9999} and compare element by element with the FP64 oracle at
|d -log10 p| <= max(1e-3, 1e-5 (-log10 p)) and |d beta| <= 1e-4 max(|beta|, se).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
from oracle.scan import decode as oracle_decode
import synth
from scan_util import compare_best, compare_full, compare_hits, oracle_panel, run_scan

pytestmark = pytest.mark.gpu

THR = 7.30103
TARGETS = (0.99, -0.99, 0.999, -0.999, 0.9999, -0.9999)


def _planted_case(encoding, N=23_000, M=200, P=16, n_cov=9, seed=123):
    """A block of M markers and a panel whose first len(TARGETS) phenotypes are planted on
    markers 10, 30, 50, ... with the target correlations; the rest are null phenotypes."""
    w = synth.Workload(f"near1_{encoding}", N=N, M=M, P=P, n_cov=n_cov, encoding=encoding,
                       missing=0.005 if encoding == "2bit" else 0.0, seed=seed, block=M,
                       causal_per_pheno=0, planted=0)
    blk = synth.make_block(w, 0)
    cov = synth.covariates(seed, N, n_cov)
    g = oracle_decode(blk["G"].numpy(), encoding, N)["g"]  # imputed, allele units
    planted = []
    rows = []
    for k, r in enumerate(TARGETS):
        j = 10 + 20 * k
        gc = g[j] - g[j].mean()
        b = math.copysign(math.sqrt(r * r / (1.0 - r * r)) * math.sqrt(N) / math.sqrt(gc @ gc), r)
        planted.append((k, torch.from_numpy(g[j]), b))
        rows.append(j)
    Yt = synth.phenotypes(seed, cov, P, planted)
    return blk, cov, Yt, rows


@pytest.mark.parametrize("precision", ["split", "fp32"])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_correlations_close_to_one_at_large_df(tgctx, encoding, precision):
    blk, cov, Yt, rows = _planted_case(encoding)
    N, P = Yt.shape[1], Yt.shape[0]
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, precision, full=True,
                       hit_mlog10p=THR)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(Yt, cov))
    assert ref["df"] >= 1500
    # the construction reached the regime it is about
    for k, (j, r) in enumerate(zip(rows, TARGETS)):
        ro = ref["r"][j, k]
        assert np.sign(ro) == np.sign(r) and 0.5 < (1 - ro * ro) / (1 - r * r) < 2.0, (k, ro, r)
    compare_full(res, ref, label=f"near1/{encoding}/{precision}")
    compare_hits(res, ref, THR)
    # the best key ranks by the FP32 product's |r|, whose rounding near |r| = 1 is relative to
    # |r| (a sum of terms of one sign): up to ~1e-5 |r| here
    worst = compare_best(res, ref, rel=1e-5)
    print(f"near1/{encoding}/{precision}: largest |r| deviation of a best key {worst:.3g}")
    got = {(int(h["marker"]), int(h["pheno"])): h for h in res["hits"]}
    for k, j in enumerate(rows):  # every planted pair is a hit with FP64-accurate statistics
        h = got[(j, k)]
        mo = ref["mlog10p"][j, k]
        assert mo > 1e4 or abs(TARGETS[k]) < 0.995
        assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (j, k, h["mlog10p"], mo)
        assert abs(h["beta"] - ref["beta"][j, k]) <= 1e-4 * max(abs(ref["beta"][j, k]), ref["se"][j, k])
        assert abs(h["se"] - ref["se"][j, k]) <= 1e-4 * ref["se"][j, k]
        assert abs(h["t"] - ref["t"][j, k]) <= 1e-5 * abs(ref["t"][j, k])
        for name in ("mlog10p", "t"):  # the FULL element near |r| = 1 agrees with the hit
            assert abs(res[name][j, k] - h[name]) <= 1e-6 * abs(h[name]) + 1e-3


@pytest.mark.parametrize("precision", ["split", "fp32"])
def test_hit_statistics_are_fp64_at_every_hit(tgctx, precision):
    """Ordinary hits (planted h^2 = 0.02 effects, -log10 p ~ 10 to 100) carry the FP64
    statistics too: with the FP32 product alone their -log10 p errors reach ~1e-4; from the FP64
    product they are within 1e-5 of the oracle's."""
    w = synth.Workload("fp64hits_u8", N=23_000, M=512, P=64, n_cov=19, encoding="u8", missing=0.0,
                       seed=31, block=512, causal_per_pheno=2)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), w.N, w.P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), w.N, w.P, "u8", precision, full=False,
                       hit_mlog10p=THR)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), "u8", oracle_panel(pan["Yt"], pan["cov_t"]))
    compare_hits(res, ref, THR)
    assert len(res["hits"]) >= 64
    for h in res["hits"]:
        j, p = int(h["marker"]), int(h["pheno"])
        mo = ref["mlog10p"][j, p]
        assert abs(h["mlog10p"] - mo) <= 1e-5 * mo + 1e-5, (j, p, h["mlog10p"], mo)
