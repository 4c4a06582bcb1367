"""Parity at the full benchmark size, N = 23,000 samples, P = 20,480 phenotypes, 20 covariate
columns, 8-bit dosages, 65,536-marker blocks, split-BF16 tensor-core scan with hit collection
(the configuration the benchmark times). The oracle recomputes sampled outputs one by one:
every hit, every planted pair, the best marker of sampled phenotypes and sampled marker norms.
A second case writes every statistic for a 256-marker block at the same N and P and compares
a sample of elements; others take the same block against small panels (the fused pass of the
scaling in P) and a 2-bit block against 2,048 phenotypes."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import r_tol, run_scan

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["n23000_m8900000_p20480_c20_u8"]
THR = 7.30103  # -log10(5e-8)


@pytest.fixture(scope="module")
def full(tgctx):
    torch.cuda.synchronize()
    pan = synth.make_panel(W, device="cuda", planted_blocks=1)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"], W.N, W.P, pan["cov_t"])
    blk = synth.make_block(W, 0, device="cuda")
    yield pan, panel, blk
    tg.tg_panel_free(panel)


def _sub_oracle(pan, blk, markers, phenos):
    """Oracle statistics for the sub-block of `markers` against the sub-panel of `phenos`."""
    Y = pan["Yt"][phenos].cpu().numpy().T.astype(np.float64)
    C = pan["cov_t"].cpu().numpy().T
    ref_panel = oracle.prepare_panel(Y, C)
    G = blk["G"][markers].cpu().numpy()
    return oracle.scan(G, "u8", ref_panel, mode="projected")


def test_fullsize_hits_planted_best_norms(tgctx, full):
    pan, panel, blk = full
    res = run_scan(tgctx, panel, blk["G"], W.N, W.P, "u8", "split", full=False, hit_mlog10p=THR,
                   hit_capacity=1 << 20)
    assert res["status"] == tg.TG_OK
    hits = res["hits"]
    assert 0 < len(hits) == res["n_hits"]
    # every planted pair is a hit
    got = {(int(h["marker"]), int(h["pheno"])) for h in hits}
    for m, p in pan["pairs"]:
        assert (m, p) in got, (m, p)
    # every hit agrees with the oracle, recomputed pair by pair
    markers = sorted({int(h["marker"]) for h in hits})
    phenos = sorted({int(h["pheno"]) for h in hits})
    ref = _sub_oracle(pan, blk, markers, phenos)
    mi = {m: i for i, m in enumerate(markers)}
    pi = {p: i for i, p in enumerate(phenos)}
    worst = {"mlog10p": 0.0, "beta_rel": 0.0}
    for h in hits:
        j, p = mi[int(h["marker"])], pi[int(h["pheno"])]
        mo = ref["mlog10p"][j, p]
        d = abs(h["mlog10p"] - mo)
        assert d <= max(1e-3, 1e-5 * mo), (h, mo)
        assert mo >= THR - max(1e-3, 1e-5 * mo)
        b, se = ref["beta"][j, p], ref["se"][j, p]
        db = abs(h["beta"] - b) / max(abs(b), se)
        assert db <= 1e-4, (h, b)
        assert abs(h["se"] - se) <= 1e-4 * se
        worst["mlog10p"] = max(worst["mlog10p"], d)
        worst["beta_rel"] = max(worst["beta_rel"], db)
    print(f"\nfull size: {len(hits)} hits, max errors vs oracle {worst}")
    # best marker of planted phenotypes is the planted marker
    for m, p in pan["pairs"][:8]:
        assert res["best_marker"][p] == m
    # marker norms for a sample of markers
    rng = np.random.default_rng(0)
    sm = np.sort(rng.choice(blk["M"], 128, replace=False))
    refm = _sub_oracle(pan, blk, sm.tolist(), [0])
    assert np.allclose(res["norm2"][sm], refm["gres2"], rtol=1e-6)
    assert np.array_equal(res["nobs"][sm], refm["decode"]["n_obs"])


def test_fullsize_best_of_a_null_phenotype(tgctx, full):
    pan, panel, blk = full
    planted = {p for _, p in pan["pairs"]}
    p0 = next(p for p in range(W.P) if p not in planted)
    res = run_scan(tgctx, panel, blk["G"], W.N, W.P, "u8", "split", full=False, hit_mlog10p=THR,
                   hit_capacity=1 << 20)
    best = -1.0
    arg = -1
    for m0 in range(0, blk["M"], 8192):
        idx = list(range(m0, min(blk["M"], m0 + 8192)))
        r = np.abs(_sub_oracle(pan, blk, idx, [p0])["r"][:, 0])
        j = int(np.nanargmax(r))
        if r[j] > best:
            best, arg = float(r[j]), m0 + j
    jg = int(res["best_marker"][p0])
    rg = abs(_sub_oracle(pan, blk, [jg], [p0])["r"][0, 0])
    tol = 2 * r_tol(W.N - W.n_cov - 2)
    assert rg >= best - tol, (jg, rg, arg, best)
    assert abs(res["best_absr"][p0] - rg) <= tol


def test_fullsize_every_statistic_sampled(tgctx, full):
    pan, panel, blk = full
    G = blk["G"][:256].contiguous()
    res = run_scan(tgctx, panel, G, W.N, W.P, "u8", "split", full=True)
    rng = np.random.default_rng(1)
    markers = np.sort(rng.choice(256, 48, replace=False)).tolist()
    phenos = np.sort(rng.choice(W.P, 300, replace=False)).tolist()
    ref = _sub_oracle(pan, {"G": G}, markers, phenos)
    for k in ("mlog10p", "beta", "se", "t"):
        sub = res[k][np.ix_(markers, phenos)]
        assert np.isfinite(sub).all()
    sub = lambda k: res[k][np.ix_(markers, phenos)]
    dm = np.abs(sub("mlog10p") - ref["mlog10p"])
    assert np.all(dm <= np.maximum(1e-3, 1e-5 * ref["mlog10p"]))
    db = np.abs(sub("beta") - ref["beta"])
    assert np.all(db <= 1e-4 * np.maximum(np.abs(ref["beta"]), ref["se"]))
    assert np.all(np.abs(sub("se") - ref["se"]) <= 1e-4 * ref["se"])
    print(f"\nfull size FULL output, sampled max errors: -log10p {dm.max():.2e}, "
          f"beta/max(|beta|,se) {(db / np.maximum(np.abs(ref['beta']), ref['se'])).max():.2e}")


W2 = synth.WORKLOADS["n23000_m1000000_p2048_c10_2bit"]


def test_2bit_panel2048_block_hits_and_sampled_statistics(tgctx):
    """2-bit calls with 0.5% missing (imputation products active), N = 23,000, P = 2,048,
    intercept + 9 covariates, one 65,536-marker block: every hit and a sample of every
    statistic against the oracle."""
    torch.cuda.synchronize()
    pan = synth.make_panel(W2, device="cuda", planted_blocks=1)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"], W2.N, W2.P, pan["cov_t"])
    try:
        blk = synth.make_block(W2, 0, device="cuda")
        res = run_scan(tgctx, panel, blk["G"], W2.N, W2.P, "2bit", "split", full=False,
                       hit_mlog10p=THR, hit_capacity=1 << 20)
        assert res["status"] == tg.TG_OK and res["n_hits"] == len(res["hits"]) > 0
        got = {(int(h["marker"]), int(h["pheno"])) for h in res["hits"]}
        for m, p in pan["pairs"]:
            assert (m, p) in got, (m, p)
        markers = sorted({int(h["marker"]) for h in res["hits"]})
        phenos = sorted({int(h["pheno"]) for h in res["hits"]})
        Y = pan["Yt"][phenos].cpu().numpy().T.astype(np.float64)
        ref = oracle.scan(blk["G"][markers].cpu().numpy(), "2bit",
                          oracle.prepare_panel(Y, pan["cov_t"].cpu().numpy().T))
        mi = {m: i for i, m in enumerate(markers)}
        pi = {p: i for i, p in enumerate(phenos)}
        worst = 0.0
        for h in res["hits"]:
            j, p = mi[int(h["marker"])], pi[int(h["pheno"])]
            mo = ref["mlog10p"][j, p]
            assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (h, mo)
            assert abs(h["beta"] - ref["beta"][j, p]) <= 1e-4 * max(abs(ref["beta"][j, p]), ref["se"][j, p])
            worst = max(worst, abs(h["mlog10p"] - mo))
        # every statistic for 256 markers, sampled against the oracle
        G = blk["G"][:256].contiguous()
        full = run_scan(tgctx, panel, G, W2.N, W2.P, "2bit", "split", full=True)
        rng = np.random.default_rng(2)
        sm = np.sort(rng.choice(256, 40, replace=False)).tolist()
        sp = np.sort(rng.choice(W2.P, 200, replace=False)).tolist()
        Y = pan["Yt"][sp].cpu().numpy().T.astype(np.float64)
        ref2 = oracle.scan(G[sm].cpu().numpy(), "2bit",
                           oracle.prepare_panel(Y, pan["cov_t"].cpu().numpy().T))
        sub = lambda k: full[k][np.ix_(sm, sp)]
        dm = np.abs(sub("mlog10p") - ref2["mlog10p"])
        assert np.all(dm <= np.maximum(1e-3, 1e-5 * ref2["mlog10p"]))
        db = np.abs(sub("beta") - ref2["beta"])
        assert np.all(db <= 1e-4 * np.maximum(np.abs(ref2["beta"]), ref2["se"]))
        print(f"\n2-bit P=2048: {len(res['hits'])} hits, max hit |d -log10 p| {worst:.2e}; "
              f"sampled max |d -log10 p| {dm.max():.2e}")
    finally:
        tg.tg_panel_free(panel)


@pytest.mark.parametrize("P", [16, 100])
def test_fullsize_small_panel_fused_pass(tgctx, full, P):
    """The small panels of the scaling in P at full size: the bench block (N = 23,000, 65,536
    8-bit dosage markers, 20 covariate columns) against P phenotypes of the full panel that
    include planted ones, so that the projection and the panel's products come from one pass
    over the packed rows with the decode fused in (P + 19 <= 64: A in tensor memory; <= 128: A
    in shared memory), which on these 256-marker tiles also writes the marker statistics. Every
    hit, the planted pairs, the best marker of the planted phenotypes, every statistic of
    sampled markers and the sampled markers' n_obs, mean and norm against the oracle."""
    pan, _, blk = full
    planted = sorted({p for _, p in pan["pairs"]})
    phenos = (planted[:P // 2] + [p for p in range(W.P) if p not in set(planted)])[:P]
    phenos = sorted(phenos)
    Yt = pan["Yt"][phenos].contiguous()
    panel = tg.tg_prepare_panel(tgctx, Yt, W.N, P, pan["cov_t"])
    try:
        res = run_scan(tgctx, panel, blk["G"], W.N, P, "u8", "split", full=True,
                       hit_mlog10p=THR, hit_capacity=1 << 20)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK and 0 < res["n_hits"] == len(res["hits"])
    col = {p: i for i, p in enumerate(phenos)}
    got = {(int(h["marker"]), int(h["pheno"])) for h in res["hits"]}
    pairs = [(m, col[p]) for m, p in pan["pairs"] if p in col]
    assert pairs
    planted_of = {}
    for m, c in pairs:
        assert (m, c) in got, (m, c)
        planted_of.setdefault(c, set()).add(m)
    for c, ms in planted_of.items():  # a phenotype's best marker is one of its planted ones
        assert int(res["best_marker"][c]) in ms, (c, res["best_marker"][c], ms)
    markers = sorted({int(h["marker"]) for h in res["hits"]})
    rng = np.random.default_rng(3)
    sm = sorted(set(markers) | set(rng.choice(blk["M"], 64, replace=False).tolist()))
    ref = _sub_oracle(pan, blk, sm, phenos)
    mi = {m: i for i, m in enumerate(sm)}
    for h in res["hits"]:
        j, c = mi[int(h["marker"])], int(h["pheno"])
        mo = ref["mlog10p"][j, c]
        assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (h, mo)
        assert abs(h["beta"] - ref["beta"][j, c]) <= 1e-4 * max(abs(ref["beta"][j, c]),
                                                                ref["se"][j, c])
    for k in ("mlog10p", "beta", "se", "t"):
        assert np.isfinite(res[k][sm]).all(), k
    dm = np.abs(res["mlog10p"][sm] - ref["mlog10p"])
    assert np.all(dm <= np.maximum(1e-3, 1e-5 * ref["mlog10p"]))
    db = np.abs(res["beta"][sm] - ref["beta"])
    assert np.all(db <= 1e-4 * np.maximum(np.abs(ref["beta"]), ref["se"]))
    assert np.all(np.abs(res["se"][sm] - ref["se"]) <= 1e-4 * ref["se"])
    assert np.array_equal(res["nobs"][sm], ref["decode"]["n_obs"])
    assert np.array_equal(res["mean"][sm], ref["decode"]["mean_units"])
    assert np.allclose(res["norm2"][sm], ref["gres2"], rtol=1e-6)
    print(f"\nfull size P={P}: {len(res['hits'])} hits, sampled max |d -log10 p| {dm.max():.2e}")
