"""The FP4 form (TG_PREC_FP4_PIECES, the low-precision multi-piece variant of the split form): 2-bit calls
exact in E2M1, the panel in six block-scaled E2M1 pieces, tcgen05 kind::mxf4 products. Compared
element by element with the FP64 oracle at the split form's tolerances; markers with a missing call
have no test in this form (NaN outputs, no hits); dosage blocks, subset panels and the static entry
point are refused."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import compare_best, compare_full, compare_hits, oracle_panel, run_scan

pytestmark = pytest.mark.gpu


def _complete_block(seed, N, M, missing_rows=()):
    """2-bit block without missing calls, except a few calls in the listed rows."""
    counts, miss = synth.hard_calls(seed, 0, synth.maf(seed, 0, M), N, 0.0)
    for j in missing_rows:
        miss[j, (7 * j) % N] = True
        miss[j, (11 * j + 3) % N] = True
    return synth.pack_2bit(counts, miss)


@pytest.mark.parametrize("mode", ["projected", "paper"])
@pytest.mark.parametrize("N,M,P", [(2001, 1000, 300), (777, 300, 40), (4100, 2051, 129)])
def test_fp4_scan_matches_oracle(tgctx, mode, N, M, P):
    cov = synth.covariates(61, N, 4)
    G = _complete_block(61, N, M, missing_rows=(3, 17, M - 1))
    Yt = synth.phenotypes(61, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    m = tg.TG_MODE_PROJECTED if mode == "projected" else tg.TG_MODE_PAPER
    try:
        res = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", "fp4", full=True, hit_mlog10p=3.0,
                       marker_offset=9, mode=m)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(G.numpy(), "2bit", oracle_panel(Yt, cov), mode=mode)
    miss_rows = np.array([3, 17, M - 1])
    # markers with a missing call: no test in the FP4 form
    assert np.isnan(res["t"][miss_rows]).all() and np.isnan(res["norm2"][miss_rows]).all()
    keep = np.setdiff1d(np.arange(M), miss_rows)
    sub = lambda d: {k: (v[keep] if isinstance(v, np.ndarray) and v.ndim == 2 else v) for k, v in d.items()}
    err = compare_full(sub(res), sub(ref), label=f"fp4/{mode}/{N}/{M}/{P}")
    print(f"fp4 {mode} N={N} M={M} P={P}: max errors vs oracle {err}")
    # hits: every GPU hit is a complete marker with oracle statistics; complete markers' hits found
    ref_keep = dict(ref)
    mlp = ref["mlog10p"].copy()
    mlp[miss_rows] = np.nan
    ref_keep["mlog10p"] = mlp
    r = ref["r"].copy()
    r[miss_rows] = np.nan
    ref_keep["r"] = r
    compare_hits(res, ref_keep, 3.0, marker_offset=9)
    compare_best(res, ref_keep, marker_offset=9)


def test_fp4_at_the_2bit_benchmark_sizes(tgctx):
    """N = 23,000, P = 2,048, intercept + 9 covariates (the 2-bit workload's panel), 4,096 complete
    markers: hits against the oracle, and every statistic of 192 markers element by element; the
    largest error per statistic is printed."""
    N, M, P = 23_000, 4096, 2048
    w = synth.WORKLOADS["n23000_m1000000_p2048_c10_2bit"]
    pan = synth.make_panel(w)
    G = _complete_block(62, N, M)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", "fp4", full=True, hit_mlog10p=6.0)
        split = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", "split", full=True, hit_mlog10p=6.0)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK and split["status"] == tg.TG_OK
    rows = np.arange(0, M, M // 192)[:192]
    ref = oracle.scan(G.numpy()[rows], "2bit", oracle_panel(pan["Yt"], pan["cov_t"]))
    sub = lambda d: {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim == 2 else v) for k, v in d.items()}
    err4 = compare_full(sub(res), ref, label="fp4 at N=23,000, P=2,048")
    err2 = compare_full(sub(split), ref, label="split at N=23,000, P=2,048")
    print(f"N=23000 P=2048 max errors vs oracle: fp4 {err4}; split {err2}")
    # the hit lists of the two forms agree up to pairs within the tolerance of the threshold
    a = {(int(h["marker"]), int(h["pheno"])): float(h["mlog10p"]) for h in res["hits"]}
    b = {(int(h["marker"]), int(h["pheno"])): float(h["mlog10p"]) for h in split["hits"]}
    for k in set(a) ^ set(b):
        v = a.get(k, b.get(k))
        assert abs(v - 6.0) <= max(1e-3, 1e-5 * v), (k, v)


def test_fp4_refuses_dosage_blocks_subset_panels_and_the_static_entry(tgctx):
    N, P = 500, 5
    cov = synth.covariates(63, N, 2)
    Yt = synth.phenotypes(63, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        D = synth.dosage_bytes(63, 0, synth.maf(63, 0, 10), N).cuda()
        opts = tg.tg_scan_opts(tg.TG_PREC_FP4_PIECES, 0, 3.0)
        out = tg.make_outputs(hits=torch.zeros(24 * 16, dtype=torch.uint8, device="cuda"),
                              n_hits=torch.zeros(1, dtype=torch.int64, device="cuda"))
        with pytest.raises(tg.TgError) as e:
            tg.tg_scan_block(tgctx, panel, D, N, 10, tg.TG_ENC_U8_DOSAGE, opts, out)
        assert e.value.status == tg.TG_ERR_UNSUPPORTED
        G = _complete_block(63, N, 10).cuda()
        with pytest.raises(tg.TgError) as e:
            tg.tg_scan_block_static(panel, G, N, 10, tg.TG_ENC_2BIT, opts, out)
        assert e.value.status == tg.TG_ERR_UNSUPPORTED
    finally:
        tg.tg_panel_free(panel)
    rows = np.ones(N, dtype=bool)
    rows[::7] = False
    from scan_util import sample_words
    sp = tg.tg_prepare_panel_subset(tgctx, Yt.cuda(), N, P, cov.cuda(), sample_words(rows).cuda())
    try:
        with pytest.raises(tg.TgError) as e:
            tg.tg_scan_block(tgctx, sp, G, N, 10, tg.TG_ENC_2BIT, opts, out)
        assert e.value.status == tg.TG_ERR_UNSUPPORTED
    finally:
        tg.tg_panel_free(sp)


def test_fp4_host_streamed_scan(tgctx):
    """tg_scan_host in the FP4 form: a complete 2-bit block streamed from pinned host memory in
    blocks that ramp up from 128 markers; the hits and per-phenotype best markers are the
    oracle's, and the same as one tg_scan_block call over the whole block."""
    from scan_util import HIT_DTYPE
    N, M, P = 2001, 3000, 300
    cov = synth.covariates(64, N, 4)
    G = _complete_block(64, N, M)
    Yt = synth.phenotypes(64, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        cap = 1 << 14
        hits_h = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        best_h = torch.zeros(P, dtype=torch.int64).pin_memory()
        opts = tg.tg_scan_opts(tg.TG_PREC_FP4_PIECES, 0, 3.0)
        nh = tg.tg_scan_host(tgctx, panel, G.pin_memory(), N, M, tg.TG_ENC_2BIT, 1024, opts,
                             hits_h, best_h, marker_offset=5)
        assert 0 < nh <= cap
        whole = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", "fp4", full=False,
                         hit_mlog10p=3.0, marker_offset=5)
    finally:
        tg.tg_panel_free(panel)
    b = best_h.numpy().view(np.uint64)
    res = {"n_hits": nh,
           "hits": np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh],
           "best_key": b,
           "best_marker": np.where(b == 0, -1, (0xFFFFFFFF - (b & 0xFFFFFFFF)).astype(np.int64)),
           "best_absr": np.frombuffer(((b >> 32).astype(np.uint32)).tobytes(), dtype=np.float32)}
    ref = oracle.scan(G.numpy(), "2bit", oracle_panel(Yt, cov))
    want, got = compare_hits(res, ref, 3.0, marker_offset=5)
    assert want > 0 and got > 0
    compare_best(res, ref, marker_offset=5)
    key = lambda h: sorted((int(x["marker"]), int(x["pheno"])) for x in h)
    assert key(res["hits"]) == key(whole["hits"])
    assert np.array_equal(b, whole["best_key"].astype(np.uint64))
