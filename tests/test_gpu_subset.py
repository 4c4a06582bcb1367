"""Panels of phenotypes observed on a subset of the samples (tg_prepare_panel_subset) against
the oracle's subset panels: the OLS of y_S on [1, C_S, g_S], genotypes imputed with their
all-sample mean, df = N_S - q - 1 (N_S - 2 in the paper's form). Phenotype values outside the
subset are NaN in every case, so a read of them would show."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import (compare_best, compare_full, compare_hits, oracle_panel, r_tol, run_scan,
                       sample_words)

pytestmark = pytest.mark.gpu

THR = 5.0


def _case(encoding, N, M, P, frac, seed, masked=False):
    w = synth.Workload(f"subset_{encoding}_{N}_{M}_{P}", N=N, M=M, P=P, n_cov=4,
                       encoding=encoding, missing=0.0 if masked else 0.02, seed=seed, block=M,
                       causal_per_pheno=2)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    miss = synth.missing_words(seed, 0, M, N, 0.03) if masked else None
    rows = np.random.default_rng(seed).random(N) < frac
    Yt = pan["Yt"].clone()
    Yt[:, torch.from_numpy(~rows)] = float("nan")
    return w, Yt, pan["cov_t"], blk, miss, rows


@pytest.mark.parametrize("encoding,masked", [("2bit", False), ("u8", True), ("u8", False)])
@pytest.mark.parametrize("precision", ["split", "fp32"])
@pytest.mark.parametrize("mode", [tg.TG_MODE_PROJECTED, tg.TG_MODE_PAPER])
def test_subset_panel_matches_oracle(tgctx, encoding, masked, precision, mode):
    w, Yt, cov, blk, miss, rows = _case(encoding, 2000, 700, 300, 0.7, 41, masked=masked)
    panel = tg.tg_prepare_panel_subset(tgctx, Yt.cuda(), w.N, w.P, cov.cuda(),
                                       sample_words(rows).cuda())
    try:
        n_used, _ = tg.tg_panel_samples(panel)
        assert n_used == rows.sum()
        df_panel = tg.tg_panel_info(panel)[3]
        res = run_scan(tgctx, panel, blk["G"].cuda(), w.N, w.P, encoding, precision, full=True,
                       hit_mlog10p=THR, missing=None if miss is None else miss.cuda(),
                       marker_offset=2, mode=mode)
        assert res["status"] == tg.TG_OK
        ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(Yt, cov, rows),
                          None if miss is None else miss.numpy(),
                          mode="paper" if mode == tg.TG_MODE_PAPER else "projected")
        assert ref["df"] == (rows.sum() - 2 if mode == tg.TG_MODE_PAPER else df_panel)
        err = compare_full(res, ref, label=f"subset {encoding}/{precision}/{mode}")
        want, got = compare_hits(res, ref, THR, marker_offset=2)
        assert want > 0 and got > 0
        compare_best(res, ref, marker_offset=2)
        ok = np.isfinite(ref["gres2"])
        assert np.array_equal(np.isfinite(res["norm2"]), ok)
        assert np.allclose(res["norm2"][ok], ref["gres2"][ok], rtol=1e-6)
        print(f"\nsubset panel ({rows.sum()} of {w.N} samples) {encoding}{'+mask' if masked else ''}/{precision}/mode {mode}: {err}")
    finally:
        tg.tg_panel_free(panel)


def test_full_subset_equals_the_plain_panel(tgctx):
    w, Yt, cov, blk, _, _ = _case("2bit", 1500, 500, 200, 1.0, 43)
    rows = np.ones(w.N, dtype=bool)
    a = tg.tg_prepare_panel_subset(tgctx, Yt.cuda(), w.N, w.P, cov.cuda(), sample_words(rows).cuda())
    b = tg.tg_prepare_panel(tgctx, Yt.cuda(), w.N, w.P, cov.cuda())
    try:
        G = blk["G"].cuda()
        ra = run_scan(tgctx, a, G, w.N, w.P, "2bit", "split", full=True, hit_mlog10p=THR)
        rb = run_scan(tgctx, b, G, w.N, w.P, "2bit", "split", full=True, hit_mlog10p=THR)
        for k in ("beta", "se", "t", "mlog10p"):
            assert np.allclose(ra[k], rb[k], rtol=1e-6, atol=1e-7, equal_nan=True), k
        assert ra["n_hits"] == rb["n_hits"]
    finally:
        tg.tg_panel_free(a)
        tg.tg_panel_free(b)


def test_missingness_groups_workflow(tgctx):
    """Phenotypes with NaN-coded missing values: masks from tg_phenotype_masks, one subset panel
    per distinct mask, panels of one mask concatenated; each group matches the oracle."""
    N, M, P = 1200, 400, 90
    cov = synth.covariates(47, N, 3)
    Yt = synth.phenotypes(47, cov, P)
    rng = np.random.default_rng(47)
    patterns = [rng.random(N) < f for f in (0.9, 0.6, 1.0)]
    group_of = rng.integers(0, 3, P)
    for p in range(P):
        Yt[p, torch.from_numpy(~patterns[group_of[p]])] = float("nan")
    Yd = Yt.cuda()
    nw = (N + 31) // 32
    masks = torch.zeros((P, nw), dtype=torch.int32, device="cuda")
    tg.tg_phenotype_masks(tgctx, Yd, N, P, masks)
    torch.cuda.synchronize()
    hm = masks.cpu().numpy()
    for p in range(P):
        assert np.array_equal(hm[p], sample_words(np.isfinite(Yt[p].numpy())).numpy())
    f = synth.maf(47, 0, M)
    counts, miss = synth.hard_calls(47, 0, f, N, 0.02)
    G = synth.pack_2bit(counts, miss)
    uniq, inv = np.unique(hm, axis=0, return_inverse=True)
    assert len(uniq) == 3
    for gi in range(len(uniq)):
        cols = np.nonzero(inv.ravel() == gi)[0]
        rows = np.isfinite(Yt[cols[0]].numpy())
        words = torch.from_numpy(uniq[gi].copy()).cuda()
        half = len(cols) // 2
        parts = [tg.tg_prepare_panel_subset(tgctx, Yd[torch.as_tensor(c, device="cuda")].contiguous(),
                                            N, len(c), cov.cuda(), words)
                 for c in (cols[:half], cols[half:])]
        panel = tg.tg_panel_concat(tgctx, parts)
        try:
            res = run_scan(tgctx, panel, G.cuda(), N, len(cols), "2bit", "split", full=True)
            ref = oracle.scan(G.numpy(), "2bit", oracle_panel(Yt[torch.as_tensor(cols)], cov, rows))
            compare_full(res, ref, label=f"group {gi}")
        finally:
            tg.tg_panel_free(panel)
            for q in parts:
                tg.tg_panel_free(q)


def test_subset_panel_rejections(tgctx):
    w, Yt, cov, blk, _, rows = _case("2bit", 800, 300, 40, 0.5, 49)
    other = ~rows
    a = tg.tg_prepare_panel_subset(tgctx, Yt.cuda(), w.N, w.P, cov.cuda(), sample_words(rows).cuda())
    Yo = Yt.clone()
    Yo[torch.isnan(Yo)] = 0.0
    b = tg.tg_prepare_panel_subset(tgctx, Yo.cuda(), w.N, w.P, cov.cuda(), sample_words(other).cuda())
    try:
        with pytest.raises(tg.TgError):
            tg.tg_panel_concat(tgctx, [a, b])
        out = tg.make_outputs(hits=torch.zeros(24, dtype=torch.uint8, device="cuda"),
                              n_hits=torch.zeros(1, dtype=torch.int64, device="cuda"))
        with pytest.raises(tg.TgError):
            tg.tg_scan_block_static(a, blk["G"].cuda(), w.N, w.M, tg.TG_ENC_2BIT,
                                    tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 0.0), out)
        few = np.zeros(w.N, dtype=bool)
        few[:2] = True
        with pytest.raises(tg.TgError):
            tg.tg_prepare_panel_subset(tgctx, Yt.cuda(), w.N, w.P, cov.cuda(), sample_words(few).cuda())
    finally:
        tg.tg_panel_free(a)
        tg.tg_panel_free(b)
