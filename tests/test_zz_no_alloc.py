"""tg_scan_block_static, the scan entry point for callers that cannot allocate device memory
(its scratch is a static device array), checked through the C ABI against tg_scan_block on
two calls in a row, and its size limit. Named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import paper_2604_21095_gb300 as tg
import synth
from scan_util import HIT_DTYPE

pytestmark = pytest.mark.gpu


def _buffers(M, P, cap=1 << 14):
    dev = "cuda"
    b = {k: torch.full((M, P), float("nan"), dtype=torch.float32, device=dev)
         for k in ("beta", "se", "t", "mlog10p")}
    b["hits"] = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    b["n_hits"] = torch.zeros(1, dtype=torch.int64, device=dev)
    b["best"] = torch.zeros(P, dtype=torch.int64, device=dev)
    b["norm2"] = torch.full((M,), float("nan"), dtype=torch.float64, device=dev)
    b["nobs"] = torch.zeros(M, dtype=torch.int32, device=dev)
    out = tg.make_outputs(beta=b["beta"], se=b["se"], t=b["t"], mlog10p=b["mlog10p"], ldo=P,
                          hits=b["hits"], n_hits=b["n_hits"], best=b["best"],
                          marker_norm2=b["norm2"], marker_nobs=b["nobs"])
    return b, out


def _host(b):
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in b.items() if k not in ("hits", "n_hits")}
    n = int(b["n_hits"].item())
    h = np.frombuffer(b["hits"].cpu().numpy().tobytes(), dtype=HIT_DTYPE)[:n]
    r["hitset"] = {(int(x["marker"]), int(x["pheno"])): x for x in h}
    return r


def _close(a, b):
    ok = np.isfinite(a["mlog10p"])
    assert np.array_equal(ok, np.isfinite(b["mlog10p"]))
    mo = b["mlog10p"][ok]
    assert np.all(np.abs(a["mlog10p"][ok] - mo) <= np.maximum(1e-3, 1e-5 * mo))
    se = b["se"][ok]
    assert np.all(np.abs(a["beta"][ok] - b["beta"][ok]) <= 1e-4 * np.maximum(np.abs(b["beta"][ok]), se))
    assert np.all(np.abs(a["se"][ok] - se) <= 1e-4 * se)
    assert set(a["hitset"]) == set(b["hitset"])
    for k, h in a["hitset"].items():
        assert abs(h["mlog10p"] - b["hitset"][k]["mlog10p"]) <= max(1e-3, 1e-5 * h["mlog10p"])
    assert np.array_equal(a["best"], b["best"])
    fin = np.isfinite(b["norm2"])
    assert np.array_equal(fin, np.isfinite(a["norm2"]))
    assert np.allclose(a["norm2"][fin], b["norm2"][fin], rtol=1e-6)
    assert np.array_equal(a["nobs"], b["nobs"])


@pytest.mark.parametrize("prec,mode", [
    (tg.TG_PREC_SPLIT_BF16, tg.TG_MODE_PROJECTED), (tg.TG_PREC_FP32, tg.TG_MODE_PROJECTED),
    (tg.TG_PREC_SPLIT_BF16, tg.TG_MODE_PAPER), (tg.TG_PREC_FP32, tg.TG_MODE_PAPER)])
@pytest.mark.parametrize("P,thr", [(300, 4.0), (40, 3.0)])  # 256- and 64-column tiles
def test_static_entry_matches_scan_block_on_two_calls_in_a_row(tgctx, P, thr, prec, mode):
    """Both precision forms (the FP32 form's operand and SIMT contraction on the static
    scratch) and both statistics (the projected OLS test, and the paper's printed form with no
    projection), on a 2-bit block and then a masked dosage block."""
    N = 1999
    cov = synth.covariates(71, N, 3)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(71, cov, P).cuda(), N, P, cov.cuda())
    try:
        counts, miss = synth.hard_calls(71, 0, synth.maf(71, 0, 700), N, 0.02)
        calls = [  # (G, encoding, missing, M) - a 2-bit block, then a masked dosage block
            (synth.pack_2bit(counts, miss).cuda(), tg.TG_ENC_2BIT, None, 700),
            (synth.dosage_bytes(71, 1, synth.maf(71, 1, 513), N).cuda(), tg.TG_ENC_U8_DOSAGE,
             synth.missing_words(71, 1, 513, N, 0.03).cuda(), 513),
        ]
        opts = tg.tg_scan_opts(prec, 1, thr, mode)
        for G, enc, missing, M in calls:
            ref_b, ref_o = _buffers(M, P)
            tg.tg_scan_block(tgctx, panel, G, N, M, enc, opts, ref_o, marker_offset=11,
                             missing=missing)
            assert tg.tg_status_poll(tgctx) == tg.TG_OK
            ref = _host(ref_b)
            got_b, got_o = _buffers(M, P)
            tg.tg_scan_block_static(panel, G, N, M, enc, opts, got_o, marker_offset=11,
                                    missing=missing)
            got = _host(got_b)
            _close(got, ref)
            assert len(ref["hitset"]) > 0
    finally:
        tg.tg_panel_free(panel)


def test_static_entry_rejects_a_block_beyond_its_scratch(tgctx):
    N, P = 23000, 4
    cov = synth.covariates(72, N, 1)
    panel = tg.tg_prepare_panel(tgctx, synth.phenotypes(72, cov, P).cuda(), N, P, cov.cuda())
    try:
        M = 4096
        G = torch.zeros(M, synth.round_up(N, 16), dtype=torch.uint8, device="cuda")
        b, out = _buffers(M, P)
        with pytest.raises(tg.TgError) as e:
            tg.tg_scan_block_static(panel, G, N, M, tg.TG_ENC_U8_DOSAGE,
                                    tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, 0.0), out)
        assert e.value.status == tg.TG_ERR_UNSUPPORTED
        assert "markers" in str(e.value)
    finally:
        tg.tg_panel_free(panel)
