"""The batched form: panels concatenated into one scan, ragged blocks replayed from one captured
CUDA graph, and autotuned kernel choice; each checked against the plain per-panel, per-block
scan (and that against the oracle elsewhere)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import HIT_DTYPE, compare_best, compare_full, oracle_panel, run_scan, sample_words

pytestmark = pytest.mark.gpu

N = 2000


def _panels(tgctx, sizes, seed=81, n_cov=3):
    cov = synth.covariates(seed, N, n_cov)
    Yt = synth.phenotypes(seed, cov, sum(sizes))
    parts, o = [], 0
    for k in sizes:
        parts.append(tg.tg_prepare_panel(tgctx, Yt[o:o + k].contiguous().cuda(), N, k, cov.cuda()))
        o += k
    return cov, Yt, parts


def test_concat_equals_each_panel_scanned_alone(tgctx):
    sizes = (17, 5, 300, 1)
    cov, Yt, parts = _panels(tgctx, sizes)
    cat = tg.tg_panel_concat(tgctx, parts)
    try:
        assert tg.tg_panel_info(cat) == (N, sum(sizes), 4, N - 5)
        counts, miss = synth.hard_calls(81, 0, synth.maf(81, 0, 700), N, 0.01)
        G = synth.pack_2bit(counts, miss).cuda()
        whole = run_scan(tgctx, cat, G, N, sum(sizes), "2bit", "split", full=True, hit_mlog10p=3.0)
        o = 0
        for part, k in zip(parts, sizes):
            alone = run_scan(tgctx, part, G, N, k, "2bit", "split", full=True, hit_mlog10p=3.0)
            for key in ("beta", "se", "t", "mlog10p"):
                assert np.array_equal(whole[key][:, o:o + k], alone[key], equal_nan=True), key
            assert np.array_equal(whole["best_key"][o:o + k], alone["best_key"])
            got = {(int(h["marker"]), int(h["pheno"]) - o) for h in whole["hits"] if o <= h["pheno"] < o + k}
            assert got == {(int(h["marker"]), int(h["pheno"])) for h in alone["hits"]}
            o += k
        ref = oracle.scan(G.cpu().numpy(), "2bit", oracle_panel(Yt, cov))
        compare_full(whole, ref, label="concatenated panel")
    finally:
        tg.tg_panel_free(cat)
        for p in parts:
            tg.tg_panel_free(p)


def test_concat_refuses_different_covariates(tgctx):
    cov_a, cov_b = synth.covariates(82, N, 2), synth.covariates(83, N, 2)
    a = tg.tg_prepare_panel(tgctx, synth.phenotypes(82, cov_a, 3).cuda(), N, 3, cov_a.cuda())
    b = tg.tg_prepare_panel(tgctx, synth.phenotypes(83, cov_b, 3).cuda(), N, 3, cov_b.cuda())
    try:
        with pytest.raises(tg.TgError) as e:
            tg.tg_panel_concat(tgctx, [a, b])
        assert e.value.status == tg.TG_ERR_INVALID_ARG
    finally:
        tg.tg_panel_free(a)
        tg.tg_panel_free(b)


def _accum_outputs(P, cap=1 << 14):
    hits = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    best = torch.zeros(P, dtype=torch.int64, device="cuda")
    return hits, n, best, tg.make_outputs(hits=hits, n_hits=n, best=best)


def _hitset(hits, n):
    h = np.frombuffer(hits.cpu().numpy().tobytes(), dtype=HIT_DTYPE)[: int(n.item())]
    return {(int(x["marker"]), int(x["pheno"])): float(x["mlog10p"]) for x in h}


@pytest.mark.parametrize("subset,P", [(False, 300), (True, 300), (False, 40)])
def test_graph_replay_equals_eager_scans_of_ragged_blocks(tgctx, subset, P):
    """Captured scans of ragged blocks replay to the eager result, for a panel of all samples,
    for a subset panel (whose marker norms come from the subset statistics kernel) and for a
    small panel (64-column tiles, split-K on these few-tile blocks, inside the capture)."""
    cov = synth.covariates(84, N, 3)
    Y = synth.phenotypes(84, cov, P).cuda()
    if subset:
        rows = np.random.default_rng(84).random(N) < 0.8
        panel = tg.tg_prepare_panel_subset(tgctx, Y, N, P, cov.cuda(), sample_words(rows).cuda())
    else:
        panel = tg.tg_prepare_panel(tgctx, Y, N, P, cov.cuda())
    ctx2 = tg.tg_create(0)  # the graph holds its context's workspace
    try:
        w = synth.Workload("ragged", N=N, M=3000, P=P, n_cov=3, encoding="2bit", missing=0.01,
                           seed=84, block=1024)
        sizes = [700, 1500, 333, 129]
        blocks = [synth.make_ragged_block(w, i, m, device="cuda") for i, m in enumerate(sizes)]
        offs = list(np.cumsum([0] + sizes[:-1]))
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 3.0)
        hits, n, best, out = _accum_outputs(P)
        for b, o in zip(blocks, offs):
            tg.tg_scan_block(tgctx, panel, b, N, b.shape[0], tg.TG_ENC_2BIT, opts, out, marker_offset=int(o))
        assert tg.tg_status_poll(tgctx) == tg.TG_OK
        eager = (_hitset(hits, n), best.cpu().numpy().copy())
        hits2, n2, best2, out2 = _accum_outputs(P)
        g = tg.tg_scan_graph_create(ctx2, panel, blocks, N, tg.TG_ENC_2BIT, opts, out2, [int(o) for o in offs])
        try:
            for _ in range(2):      # two replays from zeroed outputs give the same result
                n2.zero_()
                best2.zero_()
                tg.tg_scan_graph_launch(g)
                assert tg.tg_status_poll(ctx2) == tg.TG_OK
                got = _hitset(hits2, n2)
                assert set(got) == set(eager[0]) and len(got) > 0
                for k, v in got.items():
                    assert abs(v - eager[0][k]) <= max(1e-3, 1e-5 * v)
                assert np.array_equal(best2.cpu().numpy(), eager[1])
            # the graph holds ctx2's workspace: a larger block is refused, a smaller one scans
            big = synth.make_ragged_block(w, 9, 1600, device="cuda")
            with pytest.raises(tg.TgError) as e:
                tg.tg_scan_block(ctx2, panel, big, N, 1600, tg.TG_ENC_2BIT, opts, out2)
            assert e.value.status == tg.TG_ERR_INVALID_ARG
            tg.tg_scan_block(ctx2, panel, blocks[2], N, 333, tg.TG_ENC_2BIT, opts, out2)
            assert tg.tg_status_poll(ctx2) == tg.TG_OK
        finally:
            tg.tg_scan_graph_free(g)
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


def test_autotune_picks_a_kernel_and_results_stay_exact(tgctx):
    P = 600
    cov = synth.covariates(85, N, 3)
    Yt = synth.phenotypes(85, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    ctx2 = tg.tg_create(0)
    try:
        M = 1000
        tg.tg_autotune(ctx2, panel, tg.TG_ENC_U8_DOSAGE, M)
        choice = tg.tg_tuning(ctx2, M)
        assert choice["kernel"] in ("pair", "single") and choice["group_m"] in (4, 8, 16, 32)
        G = synth.dosage_bytes(85, 0, synth.maf(85, 0, M), N).cuda()
        res = run_scan(ctx2, panel, G, N, P, "u8", "split", full=True)
        ref = oracle.scan(G.cpu().numpy(), "u8", oracle_panel(Yt, cov))
        compare_full(res, ref, label=f"autotuned {choice}")
        compare_best(res, ref)
        print(f"\nautotuned choice for {M} markers x {P} phenotypes: {choice}")
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


@pytest.mark.parametrize("kernel,group", [("single", 8), ("single", 32), ("pair", 4), ("pair", 32)])
def test_each_tuning_choice_matches_the_oracle(tgctx, kernel, group):
    P = 257
    cov = synth.covariates(86, N, 2)
    Yt = synth.phenotypes(86, cov, P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    ctx2 = tg.tg_create(0)
    try:
        counts, miss = synth.hard_calls(86, 0, synth.maf(86, 0, 385), N, 0.01)
        G = synth.pack_2bit(counts, miss).cuda()
        tg.tg_set_tuning(ctx2, 385, kernel, group)
        assert tg.tg_tuning(ctx2, 385) == {"kernel": kernel, "group_m": group}
        ref = oracle.scan(G.cpu().numpy(), "2bit", oracle_panel(Yt, cov))
        res = run_scan(ctx2, panel, G, N, P, "2bit", "split", full=True, hit_mlog10p=3.0)
        compare_full(res, ref, label=f"{kernel}/{group}")
        compare_best(res, ref)
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


@pytest.mark.parametrize("encoding", ["2bit", "u8"])
def test_graph_with_host_blocks_equals_eager_scans(tgctx, encoding):
    """A graph whose replay copies ragged pinned host blocks to the device on a forked stream
    gives the eager scans' hits and best markers; refilled host blocks stream new markers
    through the same graph."""
    P = 300
    cov = synth.covariates(87, N, 3)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(87, cov, P).cuda(), N, P, cov.cuda())
    ctx2 = tg.tg_create(0)
    try:
        w = synth.Workload("ragged_host", N=N, M=3000, P=P, n_cov=3, encoding=encoding,
                           missing=0.01 if encoding == "2bit" else 0.0, seed=87, block=1024)
        sizes = [700, 1500, 0, 333, 129]
        offs = [int(x) for x in np.cumsum([0] + sizes[:-1])]
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 3.0)
        enc = tg.TG_ENC_2BIT if encoding == "2bit" else tg.TG_ENC_U8_DOSAGE

        def blocks_for(seed_shift):  # an empty block keeps its row stride
            return [synth.make_ragged_block(w, i + seed_shift, max(m, 1))[:m].clone()
                    for i, m in enumerate(sizes)]

        host = [b.pin_memory() for b in blocks_for(0)]
        hits2, n2, best2, out2 = _accum_outputs(P)
        g = tg.tg_scan_graph_create_host(ctx2, panel, host, N, enc, opts, out2, offs)
        try:
            for round_ in range(2):
                if round_ == 1:  # refill the pinned blocks in place: new markers, same graph
                    for h, b in zip(host, blocks_for(20)):
                        h.copy_(b)
                hits, n, best, out = _accum_outputs(P)
                for b, o in zip(host, offs):
                    if b.shape[0]:
                        tg.tg_scan_block(tgctx, panel, b.cuda(), N, b.shape[0], enc, opts, out,
                                         marker_offset=o)
                assert tg.tg_status_poll(tgctx) == tg.TG_OK
                eager = (_hitset(hits, n), best.cpu().numpy().copy())
                n2.zero_()
                best2.zero_()
                tg.tg_scan_graph_launch(g)
                assert tg.tg_status_poll(ctx2) == tg.TG_OK
                got = _hitset(hits2, n2)
                assert set(got) == set(eager[0]) and len(got) > 0
                assert np.array_equal(best2.cpu().numpy(), eager[1])
        finally:
            tg.tg_scan_graph_free(g)
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


def test_tuning_file_roundtrip(tmp_path):
    """A tuning saved to JSON loads into another context unchanged; a malformed file is refused
    and changes nothing."""
    a, b = tg.tg_create(0), tg.tg_create(0)
    try:
        tg.tg_set_tuning(a, 3000, "single", 8)
        tg.tg_set_tuning_split(a, 3000, 4)
        tg.tg_set_tuning(a, 70000, "pair", 32)
        path = tmp_path / "tuning.json"
        tg.tg_tuning_save(a, str(path))
        text = path.read_text()
        assert '"tg-tuning"' in text and '"single"' in text
        tg.tg_tuning_load(b, str(path))
        for m in (3000, 70000):
            assert tg.tg_tuning(b, m) == tg.tg_tuning(a, m)
            assert tg.tg_tuning_split(b, m) == tg.tg_tuning_split(a, m)
        bad = tmp_path / "bad.json"
        bad.write_text(text.replace('"splits": 4', '"splits": 3'))
        with pytest.raises(tg.TgError):
            tg.tg_tuning_load(b, str(bad))
        assert tg.tg_tuning_split(b, 3000) == 4  # unchanged by the refused file
        with pytest.raises(tg.TgError):
            tg.tg_tuning_load(b, str(tmp_path / "missing.json"))
    finally:
        tg.tg_destroy(a)
        tg.tg_destroy(b)


def test_second_graph_cannot_move_the_first_graphs_workspace(tgctx):
    """While a graph holds the context's buffers, another graph on the same context is accepted
    only if its blocks fit them; both then replay to the eager results."""
    P = 300
    cov = synth.covariates(88, N, 3)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(88, cov, P).cuda(), N, P, cov.cuda())
    ctx2 = tg.tg_create(0)
    try:
        w = synth.Workload("two_graphs", N=N, M=3000, P=P, n_cov=3, encoding="2bit",
                           missing=0.01, seed=88, block=1024)
        big = [synth.make_ragged_block(w, i, m, device="cuda") for i, m in enumerate([900, 700])]
        small = [synth.make_ragged_block(w, 5 + i, m, device="cuda") for i, m in enumerate([500, 300])]
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 3.0)
        h1, n1, b1, o1 = _accum_outputs(P)
        g1 = tg.tg_scan_graph_create(ctx2, panel, small, N, tg.TG_ENC_2BIT, opts, o1, [0, 500])
        try:
            h2, n2, b2, o2 = _accum_outputs(P)
            with pytest.raises(tg.TgError) as e:
                tg.tg_scan_graph_create(ctx2, panel, big, N, tg.TG_ENC_2BIT, opts, o2, [0, 900])
            assert e.value.status == tg.TG_ERR_INVALID_ARG
            g2 = tg.tg_scan_graph_create(ctx2, panel, small[1:], N, tg.TG_ENC_2BIT, opts, o2, [500])
            try:
                for g, n, b, blocks, offs in ((g1, n1, b1, small, [0, 500]),
                                              (g2, n2, b2, small[1:], [500])):
                    n.zero_()
                    b.zero_()
                    tg.tg_scan_graph_launch(g)
                    assert tg.tg_status_poll(ctx2) == tg.TG_OK
                    hits, nn, best, out = _accum_outputs(P)
                    for blk, o in zip(blocks, offs):
                        tg.tg_scan_block(tgctx, panel, blk, N, blk.shape[0], tg.TG_ENC_2BIT, opts,
                                         out, marker_offset=o)
                    assert tg.tg_status_poll(tgctx) == tg.TG_OK
                    assert np.array_equal(b.cpu().numpy(), best.cpu().numpy())
                    assert int(n.item()) == int(nn.item())
            finally:
                tg.tg_scan_graph_free(g2)
        finally:
            tg.tg_scan_graph_free(g1)
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


@pytest.mark.parametrize("encoding", ["u8", "2bit"])
def test_graph_of_small_panel_blocks_takes_the_fused_pass(tgctx, encoding):
    """A small panel (P = 16) over ragged blocks large enough for the fused joint pass: 40,000
    markers (256-marker tiles; for dosage rows the pass also writes the marker statistics),
    20,000 (128-marker tiles after a counting pass) and 1,000 (the decoded operand). Captured
    into one graph, the replay gives the eager scans' hits and best markers exactly."""
    Nf, P = 300, 16
    cov = synth.covariates(89, Nf, 3)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(89, cov, P).cuda(), Nf, P, cov.cuda())
    ctx2 = tg.tg_create(0)
    try:
        w = synth.Workload("fused_graph", N=Nf, M=61_000, P=P, n_cov=3, encoding=encoding,
                           missing=0.01 if encoding == "2bit" else 0.0, seed=89, block=40_000)
        sizes = [40_000, 20_000, 1_000]
        blocks = [synth.make_ragged_block(w, i, m, device="cuda") for i, m in enumerate(sizes)]
        offs = [int(o) for o in np.cumsum([0] + sizes[:-1])]
        enc = tg.TG_ENC_U8_DOSAGE if encoding == "u8" else tg.TG_ENC_2BIT
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 3.0)
        hits, n, best, out = _accum_outputs(P)
        for b, o in zip(blocks, offs):
            tg.tg_scan_block(tgctx, panel, b, Nf, b.shape[0], enc, opts, out, marker_offset=o)
        assert tg.tg_status_poll(tgctx) == tg.TG_OK
        eager = (_hitset(hits, n), best.cpu().numpy().copy())
        assert len(eager[0]) > 0
        hits2, n2, best2, out2 = _accum_outputs(P)
        g = tg.tg_scan_graph_create(ctx2, panel, blocks, Nf, enc, opts, out2, offs)
        try:
            for _ in range(2):
                n2.zero_()
                best2.zero_()
                tg.tg_scan_graph_launch(g)
                assert tg.tg_status_poll(ctx2) == tg.TG_OK
                got = _hitset(hits2, n2)
                assert got == eager[0]
                assert np.array_equal(best2.cpu().numpy(), eager[1])
        finally:
            tg.tg_scan_graph_free(g)
    finally:
        tg.tg_destroy(ctx2)
        tg.tg_panel_free(panel)


def test_batched_form_at_full_size(tgctx):
    """The batched form at the benchmark's sizes: the 12 panels of uneven P (8,192 phenotypes in
    all) over N = 23,000 samples with 2-bit calls (0.5% missing) and intercept + 9 covariates,
    concatenated into one panel, and the planted 65,536-marker block cut into three ragged
    blocks captured in one graph. Every planted pair is a hit, the best marker of each planted
    phenotype is one of its planted markers, and every hit matches the oracle, recomputed for the
    hits' markers and phenotypes at the scan tolerances."""
    w = synth.WORKLOADS["n23000_m500000_12panels_p8192_2bit"]
    pan = synth.make_panel(w, device="cuda", planted_blocks=1)
    ctx2 = tg.tg_create(0)  # the graph holds its context's workspace
    parts, o = [], 0
    for k in synth.BATCHED_PANELS:
        parts.append(tg.tg_prepare_panel(ctx2, pan["Yt"][o:o + k].contiguous(), w.N, k,
                                         pan["cov_t"]))
        o += k
    try:
        panel = tg.tg_panel_concat(ctx2, parts)
    finally:
        for p in parts:
            tg.tg_panel_free(p)
    try:
        G = synth.make_block(w, 0, device="cuda")["G"]
        cuts = [0, 1_537, 30_001, G.shape[0]]
        blocks = [G[a:b].contiguous() for a, b in zip(cuts, cuts[1:])]
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 7.30103)
        hits, n, best, out = _accum_outputs(w.P, cap=1 << 16)
        g = tg.tg_scan_graph_create(ctx2, panel, blocks, w.N, tg.TG_ENC_2BIT, opts, out, cuts[:-1])
        try:
            tg.tg_scan_graph_launch(g)
            assert tg.tg_status_poll(ctx2) == tg.TG_OK
        finally:
            tg.tg_scan_graph_free(g)
        got = np.frombuffer(hits.cpu().numpy().tobytes(), dtype=HIT_DTYPE)[: int(n.item())]
        assert len(got) > 0
        pairs = {(int(h["marker"]), int(h["pheno"])) for h in got}
        planted_of = {}
        for m, p in pan["pairs"]:
            assert (m, p) in pairs, (m, p)
            planted_of.setdefault(p, set()).add(m)
        bk = best.cpu().numpy().view(np.uint64)
        for p, ms in planted_of.items():
            assert int(0xFFFFFFFF - (int(bk[p]) & 0xFFFFFFFF)) in ms, p
        markers = sorted({int(h["marker"]) for h in got})
        phenos = sorted({int(h["pheno"]) for h in got})
        Y = pan["Yt"][phenos].cpu().numpy().T.astype(np.float64)
        ref = oracle.scan(G[markers].cpu().numpy(), "2bit",
                          oracle.prepare_panel(Y, pan["cov_t"].cpu().numpy().T))
        mi = {m: i for i, m in enumerate(markers)}
        pi = {p: i for i, p in enumerate(phenos)}
        for h in got:
            j, c = mi[int(h["marker"])], pi[int(h["pheno"])]
            mo = ref["mlog10p"][j, c]
            assert abs(h["mlog10p"] - mo) <= max(1e-3, 1e-5 * mo), (h, mo)
            assert abs(h["beta"] - ref["beta"][j, c]) <= 1e-4 * max(abs(ref["beta"][j, c]),
                                                                    ref["se"][j, c])
            assert abs(h["se"] - ref["se"][j, c]) <= 1e-4 * ref["se"][j, c]
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx2)
