"""The small plain workload end to end on the GPU: N = 2,000 samples, 10,000 2-bit markers with
1% missing calls, intercept + 4 covariates, 16 phenotypes with 5 planted causal markers each
(h2 = 0.02 per marker). Every (marker, phenotype) statistic is compared with the FP64 oracle for
both precision forms, the largest error of each statistic is printed, the hits at the
genome-wide threshold match, and the planted markers rank top as they do in the oracle."""
import numpy as np
import pytest

import oracle
import paper_2604_21095_gb300 as tg
import synth
from scan_util import compare_best, compare_full, compare_hits, oracle_panel, run_scan

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["n2000_m10000_p16_c5_2bit"]
GENOME_WIDE = 7.30103  # -log10(5e-8)


@pytest.fixture(scope="module")
def case():
    pan = synth.make_panel(W)
    blk = synth.make_block(W, 0)
    ref = oracle.scan(blk["G"].numpy(), "2bit", oracle_panel(pan["Yt"], pan["cov_t"]))
    return pan, blk, ref


@pytest.mark.parametrize("precision", ["split", "fp32"])
def test_small_workload_every_statistic(tgctx, case, precision):
    pan, blk, ref = case
    panel = tg.tg_prepare_panel(tgctx, pan["Yt"].cuda(), W.N, W.P, pan["cov_t"].cuda())
    try:
        res = run_scan(tgctx, panel, blk["G"].cuda(), W.N, W.P, "2bit", precision, full=True,
                       hit_mlog10p=GENOME_WIDE)
    finally:
        tg.tg_panel_free(panel)
    assert res["status"] == tg.TG_OK
    err = compare_full(res, ref, label=f"small workload/{precision}")
    want, got = compare_hits(res, ref, GENOME_WIDE)
    assert want > 0 and got > 0
    compare_best(res, ref)
    dec = ref["decode"]
    assert np.array_equal(res["nobs"], dec["n_obs"])
    assert np.array_equal(res["mean"], dec["mean_units"])
    found = found_ref = 0
    absr = np.abs(res["t"].astype(np.float64))  # |t| is monotone in |r| at fixed df
    for m, p in pan["pairs"]:
        found += m in np.argsort(-absr[:, p])[: W.causal_per_pheno]
        found_ref += m in np.argsort(-np.abs(ref["r"][:, p]))[: W.causal_per_pheno]
    assert abs(found - found_ref) <= 1 and found >= 0.9 * len(pan["pairs"])
    print(f"\nsmall workload {precision}: max |error| vs FP64 oracle per statistic {err}; "
          f"hits {got} (oracle {want}); planted markers in the top 5: {found}/{len(pan['pairs'])}")
