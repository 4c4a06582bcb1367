"""GPU parity of the whole block scan (decode, projection, contraction, epilogue) against
the FP64 oracle, for both precision forms and both genotype encodings, at sizes that span
several tiles in both directions with ragged edges, plus the degenerate cases."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import (HIT_DTYPE, compare_best, compare_full, compare_hits, enc_id, oracle_panel,
                       r_tol, run_scan)

pytestmark = pytest.mark.gpu

THR = 5.0  # hit threshold (-log10 p) for the small cases: planted effects pass it


def _case(encoding, N=2000, M=1000, P=300, n_cov=4, missing=0.01, seed=11, masked=False):
    w = synth.Workload(f"test_{encoding}_{N}_{M}_{P}", N=N, M=M, P=P, n_cov=n_cov,
                       encoding=encoding, missing=missing if not masked else 0.0, seed=seed,
                       block=M, causal_per_pheno=2)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    miss = None
    if masked:
        miss = synth.missing_words(seed, 0, M, N, missing)
    return w, pan, blk, miss


@pytest.fixture(scope="module")
def panels(tgctx):
    made = {}
    yield made
    for p in made.values():
        tg.tg_panel_free(p)


def _panel(tgctx, panels, key, pan, N, P):
    if key not in panels:
        cov = pan["cov_t"]
        panels[key] = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P,
                                          cov.cuda() if cov.shape[0] else None)
    return panels[key]


@pytest.mark.parametrize("encoding,masked", [("2bit", False), ("u8", False), ("u8", True)])
@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_scan_matches_oracle(tgctx, panels, encoding, masked, precision):
    w, pan, blk, miss = _case(encoding, masked=masked)
    panel = _panel(tgctx, panels, ("main", encoding, masked), pan, w.N, w.P)
    G = blk["G"].cuda()
    res = run_scan(tgctx, panel, G, w.N, w.P, encoding, precision, full=True, hit_mlog10p=THR,
                   missing=None if miss is None else miss.cuda(), marker_offset=7)
    assert res["status"] == tg.TG_OK
    ref_panel = oracle_panel(pan["Yt"], pan["cov_t"])
    ref = oracle.scan(blk["G"].numpy(), encoding, ref_panel,
                      None if miss is None else miss.numpy(), mode="projected")
    err = compare_full(res, ref, label=f"{encoding}/{precision}")
    want, got = compare_hits(res, ref, THR, marker_offset=7)
    assert want >= 2 * w.P * 0.5 and got > 0
    compare_best(res, ref, marker_offset=7)
    dec = ref["decode"]
    assert np.array_equal(res["nobs"], dec["n_obs"])
    assert np.array_equal(res["mean"], dec["mean_units"])
    ok = np.isfinite(ref["gres2"])
    assert np.array_equal(np.isfinite(res["norm2"]), ok)
    assert np.allclose(res["norm2"][ok], ref["gres2"][ok], rtol=1e-6)
    print(f"\nmax |error| vs FP64 oracle, {encoding}{'+mask' if masked else ''}/{precision}: {err}")


def test_scan_direct_oracle_agrees(tgctx, panels):
    """The direct-OLS oracle (the definition) on a slice of the same case."""
    w, pan, blk, _ = _case("2bit")
    panel = _panel(tgctx, panels, ("main", "2bit", False), pan, w.N, w.P)
    G = blk["G"][:64].cuda()
    res = run_scan(tgctx, panel, G, w.N, w.P, "2bit", "split", full=True)
    ref_panel = oracle_panel(pan["Yt"], pan["cov_t"])
    ref = oracle.scan(blk["G"][:64].numpy(), "2bit", ref_panel, mode="direct")
    ok = np.isfinite(ref["t"])
    assert np.all(np.abs(res["mlog10p"][ok] - ref["mlog10p"][ok]) <= np.maximum(1e-3, 1e-5 * ref["mlog10p"][ok]))
    assert np.all(np.abs(res["beta"][ok] - ref["beta"][ok]) <= 1e-4 * np.maximum(np.abs(ref["beta"][ok]), ref["se"][ok]))


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_intercept_only_is_pearson(tgctx, precision):
    """No covariates: q = 1, df = N - 2 and r is the Pearson correlation (Eq. 2, Eq. 3 as printed)."""
    N, M, P = 1999, 130, 3
    cov = synth.covariates(21, N, 0)
    Yt = synth.phenotypes(21, cov, P)
    counts, miss = synth.hard_calls(21, 0, synth.maf(21, 0, M), N, 0.0)
    G = synth.pack_2bit(counts, miss)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, None)
    try:
        assert tg.tg_panel_info(panel)[2:] == (1, N - 2)
        res = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", precision, full=True)
    finally:
        tg.tg_panel_free(panel)
    g = counts.numpy().astype(np.float64)
    y = Yt.numpy().T.astype(np.float64)
    for j in range(0, M, 13):
        for p in range(P):
            r = np.corrcoef(g[j], y[:, p])[0, 1]
            t = r * math.sqrt((N - 2) / (1 - r * r))
            assert abs(res["t"][j, p] - t) <= 2e-5 * max(1.0, abs(t))


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_degenerate_markers_and_phenotypes(tgctx, precision):
    N, M, P = 301, 9, 5
    cov = synth.covariates(31, N, 3)
    counts, miss = synth.hard_calls(31, 0, synth.maf(31, 0, M, lo=0.2), N, 0.05)
    miss[0] = True                               # every call missing
    counts[1] = 1
    miss[1] = False                              # monomorphic
    cov[2] = counts[2].double()                  # marker 2 lies in the covariate span
    miss[2] = False
    Yt = synth.phenotypes(31, cov, P)
    Yt[3] = 1.25                                 # constant phenotype
    G = synth.pack_2bit(counts, miss)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        res = run_scan(tgctx, panel, G.cuda(), N, P, "2bit", precision, full=True, hit_mlog10p=0.01)
    finally:
        tg.tg_panel_free(panel)
    for k in ("beta", "se", "t", "mlog10p"):
        assert np.isnan(res[k][:3]).all() and np.isnan(res[k][:, 3]).all()
        assert np.isfinite(res[k][3:, [0, 1, 2, 4]]).all()
    assert np.isnan(res["norm2"][:3]).all()
    assert res["nobs"][0] == 0 and np.isnan(res["mean"][0])
    for h in res["hits"]:
        assert h["marker"] >= 3 and h["pheno"] != 3
    assert res["best_marker"][3] == -1
    ref = oracle.scan(G.numpy(), "2bit", oracle_panel(Yt, cov), mode="projected")
    ok = np.isfinite(ref["r"])
    assert np.array_equal(ok, np.isfinite(res["t"]))


@pytest.mark.parametrize("precision", ["fp32", "split"])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_exact_fit_is_a_hit_with_unit_r(tgctx, precision, encoding):
    """A phenotype that is exactly b*g_j + (covariates) has |r| = 1 at marker j (r clamped to
    [-1, 1], t and -log10 p infinite or beyond any threshold, never NaN); it is the hit and the
    best marker of that phenotype with beta = b, and the other phenotypes keep oracle parity."""
    N, M, P, n_cov = 700, 40, 4, 3
    cov = synth.covariates(51, N, n_cov)
    if encoding == "2bit":
        counts, miss = synth.hard_calls(51, 0, synth.maf(51, 0, M, lo=0.2), N, 0.0)
        G = synth.pack_2bit(counts, miss)
        g = counts.double()
    else:
        G = torch.zeros(M, (N + 15) // 16 * 16, dtype=torch.uint8)  # rows padded to 16 bytes
        G[:, :N] = torch.randint(0, 256, (M, N), generator=torch.Generator().manual_seed(51),
                                 dtype=torch.uint8)
        g = G[:, :N].double() * (2.0 / 255.0)
    fits = {0: (5, 0.7), 1: (17, -1.3)}
    Yt = synth.phenotypes(51, cov, P)
    for p, (j, b) in fits.items():
        y = b * g[j] + 0.5 + cov.T @ torch.tensor([0.3, -0.2, 0.1], dtype=torch.float64)
        Yt[p] = y.float()
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        res = run_scan(tgctx, panel, G.cuda(), N, P, encoding, precision, full=True,
                       hit_mlog10p=50.0)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    for k in ("beta", "se", "t", "mlog10p"):
        assert not np.isnan(res[k]).any(), k
    got = {(int(h["marker"]), int(h["pheno"])): h for h in res["hits"]}
    for p, (j, b) in fits.items():
        h = got[(j, p)]
        assert abs(h["beta"] - b) <= 1e-4 * abs(b), (p, h["beta"], b)
        assert math.copysign(1.0, h["t"]) == math.copysign(1.0, b) and abs(h["t"]) >= 1e3
        assert h["mlog10p"] >= 1e3
        assert res["best_marker"][p] == j and res["best_absr"][p] >= 1.0 - 1e-5
        assert abs(res["t"][j, p]) >= 1e3 and res["mlog10p"][j, p] >= 1e3
        assert abs(res["beta"][j, p] - b) <= 1e-4 * abs(b)
    ref = oracle.scan(G.numpy(), encoding, oracle_panel(Yt, cov))
    keep = [2, 3]

    def sub(d):
        return {k: (v[:, keep] if isinstance(v, np.ndarray) and v.ndim == 2 else v)
                for k, v in d.items()}

    compare_full(sub(res), sub(ref), label=f"exact fit/{encoding}/{precision}")
    for p, (j, b) in fits.items():  # the oracle agrees: r = +-1 up to the FP32 rounding of Y
        assert abs(abs(ref["r"][j, p]) - 1.0) <= 1e-9 and abs(ref["beta"][j, p] - b) <= 1e-6


@pytest.mark.parametrize("M,P", [(1, 1), (129, 257), (256, 256), (5, 1000)])
@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_tile_edges(tgctx, M, P, precision):
    N = 515
    w = synth.Workload("edge", N=N, M=M, P=P, n_cov=2, encoding="u8", missing=0.0, seed=M + P, block=M)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, "u8", precision, full=True)
    finally:
        tg.tg_panel_free(panel)
    ref = oracle.scan(blk["G"].numpy(), "u8", oracle_panel(pan["Yt"], pan["cov_t"]))
    compare_full(res, ref, label=f"edge {M}x{P}/{precision}")
    compare_best(res, ref)


def test_empty_block_is_a_noop(tgctx):
    N, P = 64, 2
    cov = synth.covariates(41, N, 1)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(41, cov, P).cuda(), N, P, cov.cuda())
    try:
        G = torch.zeros(0, 16, dtype=torch.uint8, device="cuda")
        res = run_scan(tgctx, panel, G, N, P, "2bit", "split", full=False, hit_mlog10p=1.0)
        assert res["n_hits"] == 0 and res["status"] == tg.TG_OK
    finally:
        tg.tg_panel_free(panel)


def test_blocks_accumulate_hits_and_best(tgctx, panels):
    """Two half blocks with marker offsets give the same hits and best as one block."""
    w, pan, blk, _ = _case("2bit")
    panel = _panel(tgctx, panels, ("main", "2bit", False), pan, w.N, w.P)
    G = blk["G"].cuda()
    whole = run_scan(tgctx, panel, G, w.N, w.P, "2bit", "split", full=False, hit_mlog10p=THR)
    a = run_scan(tgctx, panel, G[:500], w.N, w.P, "2bit", "split", full=False, hit_mlog10p=THR)
    b = run_scan(tgctx, panel, G[500:], w.N, w.P, "2bit", "split", full=False, hit_mlog10p=THR,
                 marker_offset=500)
    key = lambda hs: sorted((int(h["marker"]), int(h["pheno"])) for h in hs)
    assert key(whole["hits"]) == sorted(key(a["hits"]) + key(b["hits"]))
    best = np.maximum(a["best_key"], b["best_key"])
    assert np.array_equal(best, whole["best_key"])


@pytest.mark.parametrize("encoding,block", [("2bit", 2048), ("u8", 1000), ("2bit", 100_000)])
def test_host_streamed_scan_matches_oracle(tgctx, panels, encoding, block):
    """tg_scan_host from pinned host memory: blocks ramp up from block/8 (256, 512, 1024, 2048
    ... for block = 2048) and the hits and best markers equal the oracle's, whatever the growth
    factor and the number of block buffers in the ring."""
    w, pan, blk, _ = _case(encoding, M=3000, P=300)
    panel = _panel(tgctx, panels, ("host", encoding), pan, w.N, w.P)
    G_host = blk["G"].pin_memory()
    cap = 1 << 14
    hits_h = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    best_h = torch.zeros(w.P, dtype=torch.int64).pin_memory()
    opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, THR)
    nh = tg.tg_scan_host(tgctx, panel, G_host, w.N, w.M, enc_id(encoding), block, opts, hits_h,
                         best_h, marker_offset=11)
    assert 0 < nh <= cap
    b = best_h.numpy().view(np.uint64)
    res = {"n_hits": nh,
           "hits": np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh],
           "best_key": b,
           "best_marker": np.where(b == 0, -1, (0xFFFFFFFF - (b & 0xFFFFFFFF)).astype(np.int64)),
           "best_absr": np.frombuffer(((b >> 32).astype(np.uint32)).tobytes(), dtype=np.float32)}
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]),
                      mode="projected")
    want, got = compare_hits(res, ref, THR, marker_offset=11)
    assert want > 0 and got > 0
    compare_best(res, ref, marker_offset=11)
    # on a fresh context (default kernel choice), later calls block by the measured copy and
    # scan times: the same hits and best markers as the first call
    ctx2 = tg.tg_create(0)
    try:
        assert tg.tg_host_ramp(ctx2) == (2.0, 0.0)  # nothing measured yet: doubling
        with pytest.raises(tg.TgError):
            tg.tg_set_host_ramp(ctx2, 0.5)
        runs = []
        for _ in range(3):
            nh2 = tg.tg_scan_host(ctx2, panel, G_host, w.N, w.M, enc_id(encoding), block, opts,
                                  hits_h, best_h, marker_offset=11)
            assert nh2 == nh
            hh = np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh2]
            runs.append((np.sort(hh, order=["marker", "pheno"]), best_h.numpy().copy()))
        assert np.array_equal(runs[0][0][["marker", "pheno"]],
                              np.sort(res["hits"], order=["marker", "pheno"])[["marker", "pheno"]])
        for hh, bb in runs[1:]:
            assert np.array_equal(hh, runs[0][0])
            assert np.array_equal(bb, runs[0][1])
        f, ratio = tg.tg_host_ramp(ctx2)
        if block < w.M:  # a second block was timed
            assert ratio > 0.0 and f == min(2.0, max(1.0, ratio))
        else:
            assert (f, ratio) == (2.0, 0.0)
        tg.tg_set_host_ramp(ctx2, 1.0)  # fixed: equal blocks of block / 8 markers
        assert tg.tg_host_ramp(ctx2)[0] == 1.0
        nh3 = tg.tg_scan_host(ctx2, panel, G_host, w.N, w.M, enc_id(encoding), block, opts,
                              hits_h, best_h, marker_offset=11)
        hh = np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh3]
        assert np.array_equal(np.sort(hh, order=["marker", "pheno"]), runs[0][0])
        # rings of 2, 4 and again 3 block buffers (shrinking frees the extra ones): the same
        for nbuf in (2, 4, 3):
            tg.tg_set_host_buffers(ctx2, nbuf)
            nh4 = tg.tg_scan_host(ctx2, panel, G_host, w.N, w.M, enc_id(encoding), block, opts,
                                  hits_h, best_h, marker_offset=11)
            hh = np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh4]
            assert np.array_equal(np.sort(hh, order=["marker", "pheno"]), runs[0][0])
            assert np.array_equal(best_h.numpy(), runs[0][1])
        for bad in (1, 5):
            with pytest.raises(tg.TgError):
                tg.tg_set_host_buffers(ctx2, bad)
    finally:
        tg.tg_destroy(ctx2)


@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_host_ring_wraps_with_many_small_blocks(tgctx, panels, encoding):
    """tg_scan_host's device ring holds host_bufs full blocks' bytes and places the blocks back
    to back, wrapping to its start. With the growth factor fixed at 1, every block of a
    block_markers = 2,048 scan has 256 markers, so 8 x host_bufs of them are in flight at once:
    5,000 markers in 20 blocks wrap a ring of two buffers (16 blocks per lap) and never reach
    the end of a ring of four. The copies run far ahead of the scans, so a block that
    overwrote bytes still being scanned would change the results: both rings give the same
    hits and best markers, bit for bit, and the same hit set as one resident scan."""
    w, pan, blk, _ = _case(encoding, M=5000, P=300)
    panel = _panel(tgctx, panels, ("ring", encoding), pan, w.N, w.P)
    G_host = blk["G"].pin_memory()
    cap = 1 << 15
    opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, THR)
    ctx2 = tg.tg_create(0)
    runs = []
    try:
        tg.tg_set_host_ramp(ctx2, 1.0)
        for nbuf in (2, 4, 2):
            tg.tg_set_host_buffers(ctx2, nbuf)
            hits_h = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
            best_h = torch.zeros(w.P, dtype=torch.int64).pin_memory()
            nh = tg.tg_scan_host(ctx2, panel, G_host, w.N, w.M, enc_id(encoding), 2048, opts,
                                 hits_h, best_h, marker_offset=3)
            assert 0 < nh <= cap
            hh = np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh]
            runs.append((np.sort(hh, order=["marker", "pheno"]), best_h.numpy().copy()))
    finally:
        tg.tg_destroy(ctx2)
    for hh, bb in runs[1:]:
        assert np.array_equal(hh, runs[0][0])
        assert np.array_equal(bb, runs[0][1])
    res = run_scan(tgctx, panel, blk["G"].cuda(), w.N, w.P, encoding, "split", full=False,
                   hit_mlog10p=THR, hit_capacity=cap, marker_offset=3)
    assert res["n_hits"] == len(runs[0][0])
    ref = np.sort(res["hits"], order=["marker", "pheno"])
    assert np.array_equal(ref[["marker", "pheno"]], runs[0][0][["marker", "pheno"]])
    assert np.allclose(ref["mlog10p"], runs[0][0]["mlog10p"], rtol=1e-5, atol=1e-4)


def test_host_streamed_edge_cases(tgctx, panels):
    """tg_scan_host at its edges, against one full call on the same context: no markers (no
    hits, best keys untouched at zero), a hit buffer smaller than the hits (the true count comes
    back, the hits written are hits of the full call, and the overflow is reported by the call
    itself, not left latched for a later status poll), no best-key buffer, and one block larger
    than the whole matrix."""
    w, pan, blk, _ = _case("2bit", M=3000, P=300)
    panel = _panel(tgctx, panels, ("host", "2bit"), pan, w.N, w.P)
    G_host = blk["G"].pin_memory()
    opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, THR)
    cap = 1 << 14

    def run(M, block, cap_, best=True):
        hits_h = torch.zeros(cap_ * HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        best_h = torch.zeros(w.P, dtype=torch.int64).pin_memory() if best else None
        nh = tg.tg_scan_host(tgctx, panel, G_host[:M], w.N, M, tg.TG_ENC_2BIT, block, opts,
                             hits_h, best_h)
        hh = np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:min(nh, cap_)]
        return nh, hh, None if best_h is None else best_h.numpy().copy()

    nh, hh, bb = run(w.M, 1024, cap)
    assert 8 < nh <= cap
    full = {(int(h["marker"]), int(h["pheno"])): h for h in hh}
    n0, h0, b0 = run(0, 1024, cap)
    assert n0 == 0 and len(h0) == 0 and not b0.any()
    n3, h3, _ = run(w.M, 1024, 3)
    assert n3 == nh and len(h3) == 3
    assert tg.tg_status_poll(tgctx) == tg.TG_OK  # the call reported its overflow and cleared it
    for h in h3:
        assert full[(int(h["marker"]), int(h["pheno"]))].tobytes() == h.tobytes()
    n4, h4, b4 = run(w.M, 1024, cap, best=False)
    assert n4 == nh and b4 is None
    assert np.array_equal(np.sort(h4, order=["marker", "pheno"]), np.sort(hh, order=["marker", "pheno"]))
    n5, h5, b5 = run(w.M, 10 * w.M, cap)
    assert n5 == nh and np.array_equal(b5, bb)
    assert set(full) == {(int(h["marker"]), int(h["pheno"])) for h in h5}


@pytest.mark.parametrize("encoding,masked", [("2bit", False), ("u8", True)])
@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_paper_mode_matches_oracle(tgctx, panels, encoding, masked, precision):
    """Eq. 2-3 as printed (marker only standardised, df = N - 2) against the oracle's paper
    form, with covariates present (where it differs from the OLS test)."""
    w, pan, blk, miss = _case(encoding, masked=masked)
    panel = _panel(tgctx, panels, ("main", encoding, masked), pan, w.N, w.P)
    G = blk["G"].cuda()
    res = run_scan(tgctx, panel, G, w.N, w.P, encoding, precision, full=True, hit_mlog10p=THR,
                   missing=None if miss is None else miss.cuda(), marker_offset=3,
                   mode=tg.TG_MODE_PAPER)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]),
                      None if miss is None else miss.numpy(), mode="paper")
    assert ref["df"] == w.N - 2
    err = compare_full(res, ref, label=f"paper {encoding}/{precision}")
    want, got = compare_hits(res, ref, THR, marker_offset=3)
    assert want > 0 and got > 0
    compare_best(res, ref, marker_offset=3)
    ok = np.isfinite(ref["gres2"])
    assert np.array_equal(np.isfinite(res["norm2"]), ok)
    assert np.allclose(res["norm2"][ok], ref["gres2"][ok], rtol=1e-10)
    # the projected statistic differs measurably with 4 covariates
    proj = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]),
                       None if miss is None else miss.numpy(), mode="projected")
    assert np.nanmax(np.abs(proj["r"] - ref["r"])) > 10 * r_tol(ref["df"])
    print(f"\nmax |error| vs FP64 oracle, paper form {encoding}/{precision}: {err}")


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_paper_mode_is_projected_mode_with_intercept_only(tgctx, precision):
    w = synth.Workload("paper_icpt", N=1500, M=700, P=130, n_cov=0, encoding="2bit",
                       missing=0.02, seed=17, block=700, causal_per_pheno=2)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), w.N, w.P, None)
    try:
        G = blk["G"].cuda()
        a = run_scan(tgctx, panel, G, w.N, w.P, "2bit", precision, full=True, hit_mlog10p=THR,
                     mode=tg.TG_MODE_PAPER)
        b = run_scan(tgctx, panel, G, w.N, w.P, "2bit", precision, full=True, hit_mlog10p=THR)
        for k in ("beta", "se", "t", "mlog10p", "best_key", "norm2"):
            assert np.array_equal(a[k], b[k], equal_nan=True), k
        assert sorted(a["hits"].tolist()) == sorted(b["hits"].tolist())
    finally:
        tg.tg_panel_free(panel)


def test_mode_argument_checked(tgctx, panels):
    w, pan, blk, _ = _case("2bit")
    panel = _panel(tgctx, panels, ("main", "2bit", False), pan, w.N, w.P)
    for opts in (tg.tg_scan_opts(1, 0, THR, 2), tg.tg_scan_opts(1, 0, THR, 0, 1)):
        out = tg.make_outputs(hits=torch.zeros(24, dtype=torch.uint8, device="cuda"),
                              n_hits=torch.zeros(1, dtype=torch.int64, device="cuda"))
        with pytest.raises(tg.TgError):
            tg.tg_scan_block(tgctx, panel, blk["G"].cuda(), w.N, w.M, tg.TG_ENC_2BIT, opts, out)


@pytest.mark.parametrize("N", [9, 33, 64, 65])
@pytest.mark.parametrize("kernel,precision", [("pair", "split"), ("single", "split"),
                                              ("pair", "fp32")])
def test_few_samples(N, kernel, precision):
    """Very small sample counts: one or two K blocks of 32 samples (a single stage of two K
    blocks, most of it zero padding), df from 6, both encodings.

    With so few samples a marker can lie close to the covariate span by chance; its r then
    carries the rounding error of the products amplified by |g_c| / |g_res| (the tolerance
    assumes a ratio near 1), so the element checks take the markers with |g_c|^2 / |g_res|^2
    <= 4 and the rest only have to agree on which results are defined. (At df = 2, p = 1 - |r|
    and no FP32-accumulated r meets an absolute 1e-3 on -log10 p near |r| = 1.)"""
    M, P = 37, 19
    ctx = tg.tg_create(0)
    try:
        tg.tg_set_tuning(ctx, M, kernel, 4)
        for encoding in ("2bit", "u8"):
            w = synth.Workload(f"few_{N}_{encoding}", N=N, M=M, P=P, n_cov=1, encoding=encoding,
                               missing=0.05 if encoding == "2bit" else 0.0, seed=N + 3, block=M)
            pan = synth.make_panel(w)
            blk = synth.make_block(w, 0)
            panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
            try:
                res = run_scan(ctx, panel, blk["G"].cuda(), N, P, encoding, precision, full=True,
                               hit_mlog10p=1.0)
            finally:
                tg.tg_panel_free(panel)
            assert res["status"] == tg.TG_OK
            ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
            assert ref["df"] == N - 3
            assert np.array_equal(np.isfinite(res["t"]), np.isfinite(ref["r"]))
            g = ref["decode"]["g"]
            gc2 = ((g - g.mean(axis=1, keepdims=True)) ** 2).sum(axis=1)
            good = np.isfinite(ref["gres2"]) & (gc2 <= 4.0 * np.nan_to_num(ref["gres2"], nan=0.0))
            assert good.sum() >= M // 2
            rows = np.nonzero(good)[0]

            def sub(d):
                return {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim == 2 else v)
                        for k, v in d.items()}

            compare_full(sub(res), sub(ref), label=f"N={N}/{encoding}/{kernel}/{precision}")
            # hits among the well-conditioned markers: the same set up to the tolerance band
            mlp = ref["mlog10p"]
            got = {(int(h["marker"]), int(h["pheno"])) for h in res["hits"] if good[h["marker"]]}
            want = {(int(j), int(q)) for j, q in zip(*np.nonzero(np.nan_to_num(mlp, nan=0.0) >= 1.0))
                    if good[j]}
            for j, q in want ^ got:
                assert abs(mlp[j, q] - 1.0) <= max(1e-3, 1e-5 * mlp[j, q]), (j, q, mlp[j, q])
    finally:
        tg.tg_destroy(ctx)


@pytest.mark.parametrize("precision", ["split", "fp32"])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_markers_close_to_the_covariate_span(tgctx, precision, encoding):
    """Covariates that nearly reproduce some markers (variance inflation |g_c|^2 / |g_res|^2 of
    about 5, 26 and 36, inside the limit of 50, and about 100, past it): the residual norms of
    such markers are recomputed in FP64 (the tensor-core projection's rounding would be
    amplified by that ratio), so the norms match the oracle to FP64 accuracy, the marker past
    the limit is NaN on both sides, and r stays within the tolerance scaled by
    sqrt(|g_c|^2 / |g_res|^2), the amplification the product itself carries."""
    N, M, P = 2000, 64, 40
    w = synth.Workload(f"collinear_{encoding}", N=N, M=M, P=P, n_cov=4, encoding=encoding,
                       missing=0.01 if encoding == "2bit" else 0.0, seed=77, block=M,
                       causal_per_pheno=1)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    dec = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))["decode"]
    g = torch.from_numpy(dec["g"])
    cov = pan["cov_t"].clone()
    noise = synth.covariates(78, N, 4)
    for k, (j, eps) in enumerate([(3, 0.5), (17, 0.2), (40, 0.17), (55, 0.1)]):
        gc = g[j] - g[j].mean()
        cov[k] = gc + eps * gc.std() * noise[k]
    Yt = synth.phenotypes(79, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, precision, full=True)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(Yt, cov))
    gc2 = ((dec["g"] - dec["g"].mean(axis=1, keepdims=True)) ** 2).sum(axis=1)
    cond = gc2 / ref["gres2"]
    assert np.nanmax(cond) > 20  # the construction reached the regime it is about
    ok = np.isfinite(ref["gres2"])
    assert not ok[55] and ok[3] and ok[17] and ok[40]  # past and inside the limit of 50
    assert np.array_equal(np.isfinite(res["norm2"]), ok)
    rel = np.abs(res["norm2"][ok] - ref["gres2"][ok]) / ref["gres2"][ok]
    refined = cond[ok] >= 2.0  # the FP64 re-projection; the rest come from the fast projection
    assert np.all(rel[refined] <= 1e-10 * cond[ok][refined]), rel[refined].max()
    assert np.all(rel[~refined] <= 1e-6), rel[~refined].max()
    df = ref["df"]
    rb = res["t"] / np.sqrt(df + res["t"].astype(np.float64) ** 2)
    dr = np.abs(rb - ref["r"])
    bound = np.broadcast_to(r_tol(df) * np.sqrt(np.maximum(cond, 1.0))[:, None], dr.shape)
    fin = np.isfinite(ref["r"])
    assert np.array_equal(np.isfinite(res["t"]), fin)
    assert np.all(dr[fin] <= bound[fin]), (dr[fin].max(), np.argmax(np.where(fin, dr / bound, 0)))


def _covariates_at_vif(g, vif, seed):
    """Covariates [N][3] (float64) such that the imputed marker g has variance inflation factor
    `vif` on [1, C] by construction: C[:, 0] = g_c + lam e with e orthogonal to 1 and g_c, the
    other two orthogonal to 1, g_c and e (they leave g's residual unchanged)."""
    r = np.random.default_rng(seed)
    N = g.size
    gc = g - g.mean()
    B = np.column_stack([np.ones(N), gc])
    e = r.standard_normal(N)
    e -= B @ np.linalg.lstsq(B, e, rcond=None)[0]
    lam = math.sqrt((gc @ gc) / (vif - 1.0) / (e @ e))
    O = r.standard_normal((N, 2))
    B3 = np.column_stack([B, e])
    O -= B3 @ np.linalg.lstsq(B3, O, rcond=None)[0]
    return np.column_stack([gc + lam * e, O])


@pytest.mark.parametrize("precision", ["split", "fp32"])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_marker_cut_matches_oracle_either_side_of_the_vif_limit(tgctx, precision, encoding):
    """A marker whose variance inflation factor on the covariates is 50 (1 - 1e-6) is tested and
    one at 50 (1 + 1e-6) is not, on the GPU as in the oracle: the NaN pattern of the norms and of
    every statistic matches the oracle's for the whole block, the other markers match within the
    usual tolerances and the tested one's r within the r tolerance scaled by sqrt(50) (the
    amplification its product carries)."""
    N, M, P, j = 2000, 64, 24, 9
    w = synth.Workload(f"vifcut_{encoding}", N=N, M=M, P=P, n_cov=3, encoding=encoding,
                       missing=0.01 if encoding == "2bit" else 0.0, seed=81, block=M,
                       causal_per_pheno=1)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    g = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))["decode"]["g"]
    for vif, tested in ((50.0 * (1 - 1e-6), True), (50.0 * (1 + 1e-6), False)):
        C = _covariates_at_vif(g[j], vif, 82)
        X = oracle.design_matrix(C, N)
        res_j = g[j] - X @ np.linalg.lstsq(X, g[j], rcond=None)[0]
        gcj = g[j] - g[j].mean()
        assert abs((gcj @ gcj) / (res_j @ res_j) / vif - 1.0) < 1e-9
        cov = torch.from_numpy(np.ascontiguousarray(C.T))
        Yt = synth.phenotypes(83, cov, P)
        panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
        try:
            res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, precision, full=True)
        finally:
            tg.tg_panel_free(panel)
        assert res["status"] == tg.TG_OK
        ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(Yt, cov))
        ok = np.isfinite(ref["gres2"])
        assert bool(ok[j]) == tested
        assert np.array_equal(np.isfinite(res["norm2"]), ok)
        assert np.array_equal(np.isfinite(res["t"]), np.isfinite(ref["r"]))
        rows = np.array([k for k in range(M) if k != j])
        compare_full({k: (v[rows] if isinstance(v, np.ndarray) and v.ndim == 2 else v) for k, v in res.items()},
                     {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim == 2 else v) for k, v in ref.items()},
                     label=f"vif {vif}/{encoding}/{precision}")
        if tested:
            df = ref["df"]
            rb = res["t"][j] / np.sqrt(df + res["t"][j].astype(np.float64) ** 2)
            assert np.all(np.abs(rb - ref["r"][j]) <= r_tol(df) * math.sqrt(50.0))


@pytest.mark.parametrize("precision", ["split", "fp32"])
def test_panel_without_phenotypes(tgctx, precision):
    """P = 0: the scan still decodes, projects and reports every marker's norm, with no hit."""
    N, M = 700, 100
    cov = synth.covariates(91, N, 2)
    counts, miss = synth.hard_calls(91, 0, synth.maf(91, 0, M), N, 0.02)
    G = synth.pack_2bit(counts, miss)
    panel = tg.tg_prepare_panel(tgctx, torch.zeros(0, N, dtype=torch.float32, device="cuda"), N, 0,
                                cov.cuda())
    try:
        assert tg.tg_panel_info(panel)[:3] == (N, 0, 3)
        res = run_scan(tgctx, panel, G.cuda(), N, 0, "2bit", precision, full=False,
                       hit_mlog10p=0.5)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK and res["n_hits"] == 0
    ref = oracle.scan(G.numpy(), "2bit", oracle_panel(synth.phenotypes(91, cov, 1), cov))
    ok = np.isfinite(ref["gres2"])
    assert np.array_equal(np.isfinite(res["norm2"]), ok)
    assert np.allclose(res["norm2"][ok], ref["gres2"][ok], rtol=1e-6)
    assert np.array_equal(res["nobs"], ref["decode"]["n_obs"])


@pytest.mark.parametrize("N", [30000, 50000, 200000])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_long_sample_axis(tgctx, N, encoding):
    """Sample counts past the one-pass decode's limits (N > 24,576 takes the row-in-registers
    kernel with twice the groups, N > 49,152 the two-pass one) and long K loops (up to 196
    accumulation chunks at a biobank-like N = 200,000), with 256-column tiles (P = 70)."""
    M, P = 200, 70
    w = synth.Workload(f"longN_{encoding}_{N}", N=N, M=M, P=P, n_cov=3, encoding=encoding,
                       missing=0.01 if encoding == "2bit" else 0.0, seed=N % 97, block=M,
                       causal_per_pheno=1)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, "split", full=True,
                       hit_mlog10p=THR)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
    compare_full(res, ref, label=f"N={N}/{encoding}")
    compare_hits(res, ref, THR)
    compare_best(res, ref)
    assert np.array_equal(res["nobs"], ref["decode"]["n_obs"])


@pytest.mark.parametrize("P,kernel,splits", [(40, "pair", 0), (300, "single", 2),
                                             (300, "single", 4), (300, "single", 1)])
@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_split_k(P, kernel, splits, encoding):
    """Blocks with fewer tiles than SMs: the one-CTA kernel splits the samples into 2 or 4
    chunk-aligned ranges (P <= 64: by rule, here 4 ranges over 5 chunks, the last one empty;
    wider panels: as tuned) and the tile's first range adds the others' partial sums in order."""
    N, M = 5000, 600
    ctx = tg.tg_create(0)
    try:
        tg.tg_set_tuning(ctx, M, kernel, 16)
        if splits:
            tg.tg_set_tuning_split(ctx, M, splits)
            assert tg.tg_tuning_split(ctx, M) == splits
        w = synth.Workload(f"splitk_{encoding}_{P}", N=N, M=M, P=P, n_cov=3, encoding=encoding,
                           missing=0.01 if encoding == "2bit" else 0.0, seed=P + 5, block=M,
                           causal_per_pheno=1)
        pan = synth.make_panel(w)
        blk = synth.make_block(w, 0)
        panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
        try:
            res = [run_scan(ctx, panel, blk["G"].cuda(), N, P, encoding, "split", full=True,
                            hit_mlog10p=THR) for _ in range(2)]
        finally:
            tg.tg_panel_free(panel)
        assert res[0]["status"] == tg.TG_OK
        for k in ("beta", "se", "t", "mlog10p"):  # the same order of additions every run
            assert np.array_equal(res[0][k], res[1][k], equal_nan=True), k
        ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
        compare_full(res[0], ref, label=f"split-K {P}/{kernel}/{splits}/{encoding}")
        compare_hits(res[0], ref, THR)
        compare_best(res[0], ref)
    finally:
        tg.tg_destroy(ctx)


@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_joint_pass_at_the_small_panel_boundaries(tgctx, encoding):
    """A panel whose phenotypes and covariate columns fit one tile (P + q - 1 <= 64, 128 or 256
    columns) gets its products from the projection's pass; one phenotype more and it goes
    through the next form (the next joint tile width, then its own contraction). Every form
    matches the oracle, and the phenotypes they share agree bit for bit."""
    N, M, n_cov = 3000, 1100, 19  # q - 1 = 19: joint tiles hold P <= 45, 109 and 237
    sizes = (45, 46, 109, 110, 237, 238)
    w = synth.Workload(f"joint_{encoding}", N=N, M=M, P=max(sizes), n_cov=n_cov,
                       encoding=encoding, missing=0.01 if encoding == "2bit" else 0.0, seed=91,
                       block=M, causal_per_pheno=1)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    cov = pan["cov_t"]
    res = {}
    for P in sizes:
        panel = tg.tg_prepare_panel(tgctx, pan["Yt"][:P].contiguous().cuda(), N, P, cov.cuda())
        try:
            res[P] = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, "split", full=True,
                              hit_mlog10p=THR)
        finally:
            tg.tg_panel_free(panel)
        assert res[P]["status"] == tg.TG_OK
        ref = oracle.scan(blk["G"].numpy(), encoding,
                          oracle_panel(pan["Yt"][:P].contiguous(), cov))
        compare_full(res[P], ref, label=f"P={P}/{encoding}")
        compare_hits(res[P], ref, THR)
        compare_best(res[P], ref)
    for a, b in zip(sizes, sizes[1:]):
        for k in ("beta", "se", "t", "mlog10p"):
            assert np.array_equal(res[a][k], res[b][k][:, :a], equal_nan=True), (a, b, k)
        assert np.array_equal(res[a]["best_key"], res[b]["best_key"][:a]), (a, b)


@pytest.mark.parametrize("P,mode", [(16, tg.TG_MODE_PROJECTED), (100, tg.TG_MODE_PROJECTED),
                                    (40, tg.TG_MODE_PAPER)])
def test_256_marker_tiles_equal_128_marker_tiles(tgctx, P, mode):
    """Blocks whose 256-marker tiles fill every SM (M >= 152 x 256) run the 64- and 128-column
    passes (the projection, a joint pass, a panel of at most 64 phenotypes) with two 128-marker
    sub-tiles per CTA sharing each B stage. The same markers scanned in two halves (128-marker
    tiles) give bit-identical statistics, and both match the oracle."""
    N, M, n_cov = 1000, 40000, 19
    w = synth.Workload(f"sub2_{P}", N=N, M=M, P=P, n_cov=n_cov, encoding="2bit", missing=0.01,
                       seed=93, block=M, causal_per_pheno=1)
    pan = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        G = blk["G"].cuda()
        whole = run_scan(tgctx, panel, G, N, P, "2bit", "split", full=True, hit_mlog10p=THR,
                         mode=mode)
        h = M // 2
        parts = [run_scan(tgctx, panel, G[o:o + h].contiguous(), N, P, "2bit", "split",
                          full=True, hit_mlog10p=THR, marker_offset=o, mode=mode)
                 for o in (0, h)]
    finally:
        tg.tg_panel_free(panel)
    assert whole["status"] == tg.TG_OK
    for k in ("beta", "se", "t", "mlog10p"):
        assert np.array_equal(whole[k], np.concatenate([parts[0][k], parts[1][k]]),
                              equal_nan=True), k
    assert np.array_equal(whole["best_key"], np.maximum(parts[0]["best_key"],
                                                        parts[1]["best_key"]))
    ref = oracle.scan(blk["G"].numpy(), "2bit", oracle_panel(pan["Yt"], pan["cov_t"]),
                      mode="projected" if mode == tg.TG_MODE_PROJECTED else "paper")
    compare_full(whole, ref, label=f"256-marker tiles P={P}")
    compare_hits(whole, ref, THR)
    compare_best(whole, ref)


@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_second_wave_of_tiles_streams_k_backwards(tgctx, encoding):
    """The CTA-pair contraction streams K from the end on the tiles of every odd wave (a wave =
    one tile per CTA pair). A block of 12,288 markers against 300 phenotypes makes 48 x 2 = 96
    tiles of 256 x 256, more than one wave on 152 SMs, so some tiles run reversed: every
    statistic is compared with the oracle, and hits and per-phenotype best keys."""
    N, M, P = 2000, 12_288, 300
    pairs = torch.cuda.get_device_properties(0).multi_processor_count // 2
    tiles = ((M + 255) // 256) * ((P + 255) // 256)
    assert pairs < tiles < 2 * pairs, (pairs, tiles)  # a second, partly reversed wave
    w, pan, blk, _ = _case(encoding, N=N, M=M, P=P, seed=17)
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), N, P, encoding, "split", full=True,
                       hit_mlog10p=THR)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    ref = oracle.scan(blk["G"].numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
    err = compare_full(res, ref, label=f"second wave/{encoding}")
    compare_hits(res, ref, THR)
    compare_best(res, ref)
    print(f"\nsecond wave of tiles ({tiles} tiles on {pairs} pairs), {encoding}: max errors {err}")
