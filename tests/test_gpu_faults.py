"""Failure detection without faulting the GPU: a bounded device wait that runs out, a hit
buffer that overflows, and arguments the library refuses before launching anything."""
import numpy as np
import pytest
import torch

import paper_2604_21095_gb300 as tg
import synth
from scan_util import run_scan

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(tgctx):
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert tg.tg_bounded_wait_test(tgctx, flag, 2_000_000) == tg.TG_ERR_TIMEOUT
    flag.fill_(1)
    assert tg.tg_bounded_wait_test(tgctx, flag, 2_000_000) == tg.TG_OK
    # the context still scans after the timeout
    N, P = 200, 3
    cov = synth.covariates(51, N, 1)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(51, cov, P).cuda(), N, P, cov.cuda())
    try:
        counts, miss = synth.hard_calls(51, 0, synth.maf(51, 0, 10), N)
        res = run_scan(tgctx, panel, synth.pack_2bit(counts, miss).cuda(), N, P, "2bit", "split")
        assert res["status"] == tg.TG_OK and np.isfinite(res["t"]).all()
    finally:
        tg.tg_panel_free(panel)


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_hit_capacity_overflow_is_reported_with_the_true_count(tgctx, precision):
    N, M, P = 400, 300, 20
    cov = synth.covariates(52, N, 1)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(52, cov, P).cuda(), N, P, cov.cuda())
    try:
        counts, miss = synth.hard_calls(52, 0, synth.maf(52, 0, M), N)
        G = synth.pack_2bit(counts, miss).cuda()
        full = run_scan(tgctx, panel, G, N, P, "2bit", precision, full=True, hit_mlog10p=0.5)
        n_true = int((full["mlog10p"] >= 0.5).sum())
        few = run_scan(tgctx, panel, G, N, P, "2bit", precision, full=False, hit_mlog10p=0.5,
                       hit_capacity=5)
    finally:
        tg.tg_panel_free(panel)
    assert abs(few["n_hits"] - n_true) <= max(3, n_true // 1000)
    assert few["n_hits"] > 5 and few["status"] == tg.TG_ERR_CAPACITY
    assert len(few["hits"]) == 5
    for h in few["hits"]:
        assert full["mlog10p"][h["marker"], h["pheno"]] >= 0.5 - 1e-3


def test_arguments_are_refused_before_launch(tgctx):
    N, P = 100, 2
    cov = synth.covariates(53, N, 1)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(53, cov, P).cuda(), N, P, cov.cuda())
    try:
        G = torch.zeros(4, 32, dtype=torch.uint8, device="cuda")
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 0.0)
        out = tg.make_outputs()
        with pytest.raises(tg.TgError) as e:      # N differs from the panel
            tg.tg_scan_block(tgctx, panel, G, N + 1, 4, tg.TG_ENC_2BIT, opts, out)
        assert e.value.status == tg.TG_ERR_INVALID_ARG
        G26 = torch.zeros(4, 26, dtype=torch.uint8, device="cuda")
        with pytest.raises(tg.TgError) as e:      # row stride not a multiple of 16
            tg.tg_scan_block(tgctx, panel, G26, N, 4, tg.TG_ENC_2BIT, opts, out)
        assert e.value.status == tg.TG_ERR_INVALID_ARG
        with pytest.raises(tg.TgError) as e:      # 2-bit calls with an external mask
            tg.tg_scan_block(tgctx, panel, G, N, 4, tg.TG_ENC_2BIT, opts, out,
                             missing=torch.zeros(4, 4, dtype=torch.int32, device="cuda"))
        assert e.value.status == tg.TG_ERR_INVALID_ARG
        with pytest.raises(tg.TgError) as e:      # dosage rows shorter than N
            tg.tg_scan_block(tgctx, panel, G, N, 4, tg.TG_ENC_U8_DOSAGE, opts, out)
        assert e.value.status == tg.TG_ERR_INVALID_ARG
        bad = tg.tg_scan_opts(7, 0, 0.0)
        with pytest.raises(tg.TgError):
            tg.tg_scan_block(tgctx, panel, G, N, 4, tg.TG_ENC_2BIT, bad, out)
        assert tg.tg_status_poll(tgctx) == tg.TG_OK
    finally:
        tg.tg_panel_free(panel)


def test_allocation_failure_is_reported_and_the_context_survives(tgctx):
    """Host-side fault injection by size: a panel and a block whose device buffers cannot be
    allocated (hundreds of GB) give TG_ERR_OOM before any kernel reads the inputs; the same
    context then prepares and scans normally. The oversized block is declared with far more rows
    than its buffer holds, so it must fail in the decoded operand's allocation, before any
    kernel: fused decoding (which needs no operand buffer) is off for that call."""
    N, P = 23000, 3
    cov = synth.covariates(53, N, 1)
    Y = synth.phenotypes(53, cov, P).cuda()
    with pytest.raises(tg.TgError) as e:  # Y_res alone would need P * N * 8 = 736 GB
        tg.tg_prepare_panel(tgctx, Y[:1], N, 4_000_000, cov.cuda())
    assert e.value.status == tg.TG_ERR_OOM
    panel = tg.tg_prepare_panel(tgctx, Y, N, P, cov.cuda())
    try:
        counts, miss = synth.hard_calls(53, 0, synth.maf(53, 0, 64), N)
        G = synth.pack_2bit(counts, miss).cuda()
        huge_M = 20_000_000  # the decoded operand alone would need huge_M * 23,040 * 2 = 920 GB
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 7.3)
        n_hits = torch.zeros(1, dtype=torch.int64, device="cuda")
        hits = torch.zeros(24 * 16, dtype=torch.uint8, device="cuda")
        out = tg.make_outputs(hits=hits, n_hits=n_hits)
        tg.tg_set_fused_decode(tgctx, tg.TG_FUSED_OFF)
        try:
            with pytest.raises(tg.TgError) as e:
                tg.tg_scan_block(tgctx, panel, G, N, huge_M, tg.TG_ENC_2BIT, opts, out)
        finally:
            tg.tg_set_fused_decode(tgctx, tg.TG_FUSED_SMALL_PANELS)
        assert e.value.status == tg.TG_ERR_OOM
        res = run_scan(tgctx, panel, G, N, P, "2bit", "split")
        assert res["status"] == tg.TG_OK and np.isfinite(res["t"]).all()
    finally:
        tg.tg_panel_free(panel)
