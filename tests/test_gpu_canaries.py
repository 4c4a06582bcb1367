"""Out-of-bounds writes, checked without a sanitizer: every output buffer is allocated larger than
the call's sizes and filled with a canary, and after the scan everything past the sizes the call
was given must still hold the canary. Covers both precisions, both tensor-core kernels, 64-column
tiles with split-K, ragged sizes and a hit buffer that overflows."""
import numpy as np
import pytest
import torch

import paper_2604_21095_gb300 as tg
import synth
from scan_util import HIT_DTYPE

pytestmark = pytest.mark.gpu

CANARY_F = 1234.5
CANARY_I = -77
CANARY_B = 0xA5


@pytest.mark.parametrize("P,kernel,precision", [(300, "pair", "split"), (300, "single", "split"),
                                                (40, "single", "split"), (257, "pair", "fp32")])
@pytest.mark.parametrize("M", [129, 1000])
def test_outputs_are_written_only_within_their_sizes(M, P, kernel, precision):
    N, ldo, cap, pad = 1999, P + 7, 64, 5
    dev = "cuda"
    cov = synth.covariates(61, N, 3)
    ctx = tg.tg_create(0)
    panel = tg.tg_prepare_panel(ctx, synth.phenotypes(61, cov, P).cuda(), N, P, cov.cuda())
    try:
        tg.tg_set_tuning(ctx, M, kernel, 8)
        counts, miss = synth.hard_calls(61, 0, synth.maf(61, 0, M), N, 0.02)
        G = synth.pack_2bit(counts, miss).cuda()
        full = {k: torch.full((M + pad, ldo), CANARY_F, dtype=torch.float32, device=dev)
                for k in ("beta", "se", "t", "mlog10p")}
        hits = torch.full(((cap + 16) * HIT_DTYPE.itemsize,), CANARY_B, dtype=torch.uint8,
                          device=dev)
        n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
        best = torch.full((P + 8,), CANARY_I, dtype=torch.int64, device=dev)
        best[:P] = 0
        norm2 = torch.full((M + pad,), CANARY_F, dtype=torch.float64, device=dev)
        nobs = torch.full((M + pad,), CANARY_I, dtype=torch.int32, device=dev)
        mean = torch.full((M + pad,), CANARY_F, dtype=torch.float64, device=dev)
        out = tg.make_outputs(beta=full["beta"], se=full["se"], t=full["t"],
                              mlog10p=full["mlog10p"], ldo=ldo, hits=hits, n_hits=n_hits,
                              best=best, marker_norm2=norm2, marker_nobs=nobs, marker_mean=mean)
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16 if precision == "split" else tg.TG_PREC_FP32,
                               1, 1.0)  # a low threshold: the hit buffer overflows
        out.hit_capacity = cap  # the buffer holds 16 records more: they must stay untouched
        tg.tg_scan_block(ctx, panel, G, N, M, tg.TG_ENC_2BIT, opts, out)
        status = tg.tg_status_poll(ctx)
        torch.cuda.synchronize()
        assert status == tg.TG_ERR_CAPACITY and int(n_hits.item()) > cap
        for k, v in full.items():
            h = v.cpu().numpy()
            assert np.all(h[:M, P:] == CANARY_F), k     # columns past P
            assert np.all(h[M:] == CANARY_F), k         # rows past M
            assert not np.any(h[:M, :P] == CANARY_F), k  # every element written
        hb = hits.cpu().numpy()
        assert np.all(hb[cap * HIT_DTYPE.itemsize:] == CANARY_B)
        bb = best.cpu().numpy()
        assert np.all(bb[P:] == CANARY_I)
        for v, c in ((norm2, CANARY_F), (nobs, CANARY_I), (mean, CANARY_F)):
            h = v.cpu().numpy()
            assert np.all(h[M:] == c)
            assert not np.any(h[:M] == c)
    finally:
        tg.tg_panel_free(panel)
        tg.tg_destroy(ctx)
