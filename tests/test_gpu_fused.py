"""Decoding the genotypes inside the contraction kernels (tg_set_fused_decode, for split-form
2-bit blocks and unmasked dosage blocks) against the default path that first writes the
decoded operand to device memory: every output must be bit-identical, for both kernels (CTA
pairs and one CTA per tile), both encodings, sample counts that end inside a K block and blocks
whose last m-tiles are partly or wholly past M, and small panels whose products come from the
projection's pass (64-, 128- and 256-column joint tiles). The fused path is also compared with
the FP64 oracle directly, element by element at the scan tolerances."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import compare_best, compare_full, compare_hits, oracle_panel, run_scan

pytestmark = pytest.mark.gpu


def _outputs_equal(a, b):
    for k in ("beta", "se", "t", "mlog10p", "best_key", "norm2", "nobs", "mean"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    key = lambda r: sorted(tuple(h) for h in r["hits"].tolist())
    assert a["n_hits"] == b["n_hits"] and key(a) == key(b)


@pytest.mark.parametrize("encoding", ["2bit", "u8"])
@pytest.mark.parametrize("kernel", ["pair", "single"])
@pytest.mark.parametrize("N,M,P", [(2000, 1000, 300), (1999, 777, 513), (257, 300, 40),
                                   (23000, 520, 600), (2000, 1000, 100), (1999, 777, 230)])
def test_fused_decode_is_bit_identical(encoding, kernel, N, M, P):
    w = synth.Workload(f"fused_{encoding}_{N}_{M}_{P}", N=N, M=M, P=P, n_cov=4,
                       encoding=encoding, missing=0.03 if encoding == "2bit" else 0.0, seed=29,
                       block=M, causal_per_pheno=1)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0)["G"].cuda()
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        tg.tg_set_tuning(ctx, M, kernel, 4)
        res = {}
        for fused in (True, False):
            tg.tg_set_fused_decode(ctx, fused)
            res[fused] = run_scan(ctx, panel, G, N, P, encoding, "split", full=True,
                                  hit_mlog10p=3.0, marker_offset=5)
            assert res[fused]["status"] == tg.TG_OK
        assert res[True]["n_hits"] > 0
        _outputs_equal(res[True], res[False])
        ref = oracle.scan(G.cpu().numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
        compare_full(res[True], ref, label=f"fused/{encoding}/{kernel}/{N}/{M}/{P}")
        compare_hits(res[True], ref, 3.0, marker_offset=5)
        compare_best(res[True], ref, marker_offset=5)
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)


@pytest.mark.parametrize("encoding,N,M,P", [
    ("2bit", 1999, 39_000, 40),   # joint operand of 64 rows, 256-marker tiles
    ("u8", 2000, 39_000, 100),    # 128 rows, 256-marker tiles (one pass: no counting pass)
    ("u8", 1999, 39_000, 40),     # 64 rows, 256-marker tiles (one pass)
    ("u8", 45, 39_000, 16),       # one pass with N < 64: the shift from fewer samples
    ("2bit", 2001, 20_000, 100),  # 128 rows, 128-marker tiles
    ("u8", 1999, 20_000, 40),     # 64 rows, 128-marker tiles
])
def test_fused_joint_pass_of_small_panels(encoding, N, M, P):
    """The joint projection pass of a small panel that decodes the packed rows in shared memory
    (the default for such panels and blocks) against the FP64 oracle and the decoded-operand
    path, with sample counts that end inside a K block and a last tile that is partly past M.
    2-bit calls take the same bf16 values as the decoded operand, so their results are
    bit-identical to it; dosage bytes are expanded into f16 against an f16 hi + lo joint operand
    (a different split of the panel), so both paths are held to the oracle's tolerances. On
    256-marker tiles the dosage pass also writes the marker statistics itself (no counting pass
    runs first): n_obs and the mean must equal the counting pass's bit for bit, with the bytes
    past N in each row set to nonzero padding that neither path may count."""
    w = synth.Workload(f"fusedjoint_{encoding}_{N}_{M}_{P}", N=N, M=M, P=P, n_cov=4,
                       encoding=encoding, missing=0.02 if encoding == "2bit" else 0.0, seed=43,
                       block=M, causal_per_pheno=1)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0)["G"].cuda()
    if encoding == "u8" and G.shape[1] > N:
        G[:, N:] = 0xAB  # row padding: not samples
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = {}
        for setting in (tg.TG_FUSED_SMALL_PANELS, tg.TG_FUSED_OFF):
            tg.tg_set_fused_decode(ctx, setting)
            res[setting] = run_scan(ctx, panel, G, N, P, encoding, "split", full=True,
                                    hit_mlog10p=4.0, marker_offset=3)
            assert res[setting]["status"] == tg.TG_OK
        got = res[tg.TG_FUSED_SMALL_PANELS]
        if encoding == "2bit":
            _outputs_equal(got, res[tg.TG_FUSED_OFF])
        else:
            for k in ("nobs", "mean"):
                assert np.array_equal(got[k], res[tg.TG_FUSED_OFF][k]), k
        assert got["n_hits"] > 0
        ref = oracle.scan(G.cpu().numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
        for setting, r in res.items():
            compare_full(r, ref, label=f"fused joint {setting}/{encoding}/{N}/{M}/{P}")
            compare_hits(r, ref, 4.0, marker_offset=3)
            compare_best(r, ref, marker_offset=3)
            assert np.array_equal(r["nobs"], ref["decode"]["n_obs"])
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)


@pytest.mark.parametrize("encoding,N,M,P", [
    ("2bit", 1999, 39_000, 300),  # 256-marker tiles after a counting pass
    ("u8", 2000, 39_000, 300),    # 256-marker tiles, one pass (no counting pass)
    ("u8", 45, 39_000, 200),      # one pass with N < 64; a panel that had a 256-row joint operand
    ("2bit", 2001, 20_000, 300),  # 128-marker tiles
    ("u8", 1999, 39_000, 150),    # one pass; a 256-row joint operand's panel
    ("u8", 1999, 20_000, 513),    # 128-marker tiles after a counting pass
    ("2bit", 2001, 39_000, 150),  # a 256-row joint operand with a counting pass: the joint pass
])
def test_fused_projection_pass_writes_the_operand(encoding, N, M, P):
    """A panel too large for the joint pass (P + q - 1 > 128): its projection runs as the same
    pass over the packed rows with the projection columns alone, which also writes the block's
    operand for the panel's contraction. Against the FP64 oracle and the decoded-operand path.
    2-bit calls expand to the decoded operand's bf16 values and the projection reads the same
    bf16 projection columns, so the two paths agree bit for bit. (A panel with a 256-row joint
    operand, P + q - 1 <= 256, takes this pass only where the pass writes the statistics, dosage
    rows on 256-marker tiles; 2-bit blocks keep its one joint pass.) Dosage rows take the f16
    projection columns (and, on 256-marker tiles, each row's shift from its first 64 bytes, the
    statistics written by the pass), so they are held to the oracle's tolerances, with n_obs and
    the mean equal to the counting pass's and nonzero padding past N in every row."""
    w = synth.Workload(f"fusedproj_{encoding}_{N}_{M}_{P}", N=N, M=M, P=P, n_cov=4,
                       encoding=encoding, missing=0.02 if encoding == "2bit" else 0.0, seed=53,
                       block=M, causal_per_pheno=1)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0)["G"].cuda()
    if encoding == "u8" and G.shape[1] > N:
        G[:, N:] = 0xAB  # row padding: not samples
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = {}
        for setting in (tg.TG_FUSED_SMALL_PANELS, tg.TG_FUSED_OFF):
            tg.tg_set_fused_decode(ctx, setting)
            res[setting] = run_scan(ctx, panel, G, N, P, encoding, "split", full=True,
                                    hit_mlog10p=4.0, marker_offset=7)
            assert res[setting]["status"] == tg.TG_OK
        got = res[tg.TG_FUSED_SMALL_PANELS]
        if encoding == "2bit":
            _outputs_equal(got, res[tg.TG_FUSED_OFF])
        else:
            for k in ("nobs", "mean"):
                assert np.array_equal(got[k], res[tg.TG_FUSED_OFF][k]), k
        assert got["n_hits"] > 0
        ref = oracle.scan(G.cpu().numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
        for setting, r in res.items():
            compare_full(r, ref, label=f"fused projection {setting}/{encoding}/{N}/{M}/{P}")
            compare_hits(r, ref, 4.0, marker_offset=7)
            compare_best(r, ref, marker_offset=7)
            assert np.array_equal(r["nobs"], ref["decode"]["n_obs"])
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)


def test_masked_dosage_blocks_use_the_decoded_operand():
    """A dosage block with a missing mask is scanned through the decoded operand whatever the
    setting; the result does not depend on it."""
    w = synth.Workload("fused_masked", N=1500, M=600, P=200, n_cov=2, encoding="u8",
                       missing=0.0, seed=31, block=600, causal_per_pheno=1)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0)["G"].cuda()
    miss = synth.missing_words(31, 0, w.M, w.N, 0.05).cuda()
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), w.N, w.P, pan["cov_t"].cuda())
    try:
        res = {}
        for fused in (True, False):
            tg.tg_set_fused_decode(ctx, fused)
            res[fused] = run_scan(ctx, panel, G, w.N, w.P, "u8", "split", full=True,
                                  hit_mlog10p=3.0, missing=miss)
        _outputs_equal(res[True], res[False])
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)


@pytest.mark.parametrize("encoding", ["u8", "2bit"])
def test_host_streamed_small_panel_mixes_the_paths(encoding):
    """tg_scan_host with a small panel (P = 16): its blocks ramp up from 8,192 markers, so the
    first go through the decoded operand and the later ones through the fused joint pass (on
    128- and then 256-marker tiles; for dosage rows the latter writes the marker statistics
    itself). The hits and best markers of the whole stream are the oracle's."""
    from scan_util import HIT_DTYPE
    N, M, P = 300, 100_000, 16
    w = synth.Workload(f"fused_host_{encoding}", N=N, M=M, P=P, n_cov=3, encoding=encoding,
                       missing=0.01 if encoding == "2bit" else 0.0, seed=47, block=M,
                       causal_per_pheno=2)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0)["G"]
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        sizes = tg.tg_host_block_sizes(M, 65_536, tg.tg_host_ramp(ctx)[0])
        assert sizes[0] < 128 * 152 and max(sizes) >= 256 * 152  # both routes are taken
        cap = 1 << 16
        hits_h = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        best_h = torch.zeros(P, dtype=torch.int64).pin_memory()
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 4.0)
        nh = tg.tg_scan_host(ctx, panel, G.pin_memory(), N, M,
                             tg.TG_ENC_U8_DOSAGE if encoding == "u8" else tg.TG_ENC_2BIT,
                             65_536, opts, hits_h, best_h)
        assert 0 < nh <= cap
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)
    b = best_h.numpy().view(np.uint64)
    res = {"n_hits": nh,
           "hits": np.frombuffer(hits_h.numpy().tobytes(), dtype=HIT_DTYPE)[:nh],
           "best_key": b,
           "best_marker": np.where(b == 0, -1, (0xFFFFFFFF - (b & 0xFFFFFFFF)).astype(np.int64)),
           "best_absr": np.frombuffer(((b >> 32).astype(np.uint32)).tobytes(), dtype=np.float32)}
    ref = oracle.scan(G.numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
    want, got = compare_hits(res, ref, 4.0)
    assert want > 0 and got > 0
    compare_best(res, ref)


@pytest.mark.parametrize("encoding,N", [("u8", 70_000), ("2bit", 100_000)])
def test_fused_joint_pass_at_a_long_sample_axis(encoding, N):
    """The fused joint pass of a small panel (P = 40, 256-marker tiles) at biobank-like sample
    counts: dosage rows beyond the one-pass limit (N > 66,051, where the sum of squared bytes
    would overflow 32 bits) take a counting pass first, as 2-bit rows always do, and both run
    hundreds of 64-sample stages per tile. Every hit and every statistic of sampled markers
    against the oracle, recomputed for those markers; n_obs and the mean exact."""
    M, P = 39_000, 40
    w = synth.Workload(f"fusedlong_{encoding}_{N}", N=N, M=M, P=P, n_cov=4, encoding=encoding,
                       missing=0.01 if encoding == "2bit" else 0.0, seed=61, block=M,
                       causal_per_pheno=1)
    pan = synth.make_panel(w)
    G = synth.make_block(w, 0, device="cuda")["G"]
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, pan["Yt"].cuda(), N, P, pan["cov_t"].cuda())
    try:
        res = run_scan(ctx, panel, G, N, P, encoding, "split", full=True, hit_mlog10p=5.0,
                       hit_capacity=1 << 16)
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)
    assert res["status"] == tg.TG_OK and res["n_hits"] > 0
    rng = np.random.default_rng(5)
    sm = sorted({int(h["marker"]) for h in res["hits"]} | set(rng.choice(M, 48, replace=False).tolist()))
    ref = oracle.scan(G[sm].cpu().numpy(), encoding, oracle_panel(pan["Yt"], pan["cov_t"]))
    sub = {k: res[k][sm] for k in ("beta", "se", "t", "mlog10p", "nobs", "mean", "norm2")}
    compare_full(sub, ref, label=f"fused joint N={N}/{encoding}")
    mi = {m: i for i, m in enumerate(sm)}
    for h in res["hits"]:
        mo = ref["mlog10p"][mi[int(h["marker"])], int(h["pheno"])]
        assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (h, mo)
    assert np.array_equal(sub["nobs"], ref["decode"]["n_obs"])
    assert np.array_equal(sub["mean"], ref["decode"]["mean_units"])
