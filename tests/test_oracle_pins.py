"""Pins of the FP64 oracle against things other than itself.

Closed forms, brute force on tiny inputs, an arbitrary-precision library, published
table values and invariants of the OLS test. No GPU is used here.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import decode as odec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- decode

def test_plink_bed_golden_bytes():
    rows = []
    for line in open(os.path.join(GOLDEN, "plink_bed_bytes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        b, *vals = line.split()
        rows.append((int(b, 16), vals))
    G = np.array([[b for b, _ in rows]], dtype=np.uint8)
    counts, miss = oracle.decode_2bit(G, 4 * len(rows))
    for k, (_, vals) in enumerate(rows):
        for s, v in enumerate(vals):
            i = 4 * k + s
            if v == "NA":
                assert miss[0, i]
            else:
                assert not miss[0, i] and counts[0, i] == int(v)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 37, 64, 130])
def test_pack_decode_roundtrip(N):
    g = torch.Generator().manual_seed(N)
    counts = torch.randint(0, 3, (9, N), generator=g, dtype=torch.int8)
    miss = torch.rand(9, N, generator=g) < 0.2
    G = synth.pack_2bit(counts, miss).numpy()
    assert G.shape[1] % 16 == 0
    c, m = oracle.decode_2bit(G, N)
    assert np.array_equal(m, miss.numpy())
    assert np.array_equal(np.where(m, 0, c), np.where(miss.numpy(), 0, counts.numpy()))


def test_all_256_bytes_against_field_table():
    G = np.arange(256, dtype=np.uint8)[:, None]
    c, m = oracle.decode_2bit(G, 4)
    table = {0b00: 2, 0b10: 1, 0b11: 0}
    for b in range(256):
        for s in range(4):
            f = (b >> (2 * s)) & 3
            assert m[b, s] == (f == 0b01)
            if f != 0b01:
                assert c[b, s] == table[f]


def test_marker_stats_exact_and_correctly_rounded():
    r = _rng(3)
    units = r.integers(0, 256, size=(40, 301))
    miss = r.random((40, 301)) < 0.3
    miss[0] = True               # no observed call
    miss[1] = False
    n, S, S2, mean = oracle.marker_stats(units, miss)
    for j in range(40):
        obs = [int(u) for u, mm in zip(units[j], miss[j]) if not mm]
        assert n[j] == len(obs) and S[j] == sum(obs) and S2[j] == sum(u * u for u in obs)
        if obs:
            assert mean[j] == float(Fraction(sum(obs), len(obs)))
        else:
            assert np.isnan(mean[j])


def test_u8_mask_and_imputation():
    r = _rng(4)
    N = 70
    G = r.integers(0, 256, size=(5, 80)).astype(np.uint8)
    miss = r.random((5, N)) < 0.25
    words = np.zeros((5, 3), dtype=np.int64)
    for j in range(5):
        for i in range(N):
            if miss[j, i]:
                words[j, i // 32] |= 1 << (i % 32)
    words = np.where(words >= 2 ** 31, words - 2 ** 32, words).astype(np.int32)
    units, m = oracle.decode_u8(G, N, words)
    assert np.array_equal(m, miss)
    n, S, S2, mean = oracle.marker_stats(units, m)
    g = oracle.impute(units, m, mean, odec.DOSAGE_SCALE)
    for j in range(5):
        obs = G[j, :N][~miss[j]].astype(float)
        assert np.allclose(g[j][~miss[j]], obs * 2 / 255)
        assert np.allclose(g[j][miss[j]], obs.mean() * 2 / 255)


def test_synth_mask_words_match_bits():
    w = synth.missing_words(9, 0, 6, 70, 0.3)
    m = odec.unpack_mask(w.numpy(), 6, 70)
    assert 0.15 < m.mean() < 0.45
    # bit i%32 of word i//32
    j, i = np.argwhere(m)[0]
    assert (int(w[j, i // 32]) >> (i % 32)) & 1 == 1


# ---------------------------------------------------------------- panel

def test_householder_basis_orthonormal_and_spans_X():
    r = _rng(5)
    N = 60
    X = oracle.design_matrix(r.standard_normal((N, 5)), N)
    Q, kept = oracle.householder_basis(X)
    assert kept == list(range(6))
    assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-13)
    Pq = Q @ Q.T
    Px = X @ np.linalg.pinv(X)
    assert np.allclose(Pq, Px, atol=1e-12)
    Qn, _ = np.linalg.qr(X)
    assert np.allclose(Pq, Qn @ Qn.T, atol=1e-12)
    # first column spans the intercept
    assert np.allclose(np.abs(Q[:, 0]), 1 / math.sqrt(N))


def test_householder_rank_detection():
    r = _rng(6)
    N = 40
    C = r.standard_normal((N, 4))
    C = np.column_stack([C, C[:, 1], np.full(N, 3.0), 2 * C[:, 0] - C[:, 3]])
    X = oracle.design_matrix(C, N)
    Q, kept = oracle.householder_basis(X)
    assert kept == [0, 1, 2, 3, 4]
    assert Q.shape == (N, 5)
    assert np.allclose(X @ np.linalg.pinv(X), Q @ Q.T, atol=1e-10)


def test_residualise_against_lstsq():
    r = _rng(7)
    N, P = 80, 6
    C = r.standard_normal((N, 3))
    X = oracle.design_matrix(C, N)
    Y = X @ r.standard_normal((4, P)) + r.standard_normal((N, P))
    Y[:, 4] = 2.5                      # constant phenotype
    Y[:, 5] = C[:, 1] * 3.0 - 1.0      # inside the covariate span
    Q, _ = oracle.householder_basis(X)
    Yres, s, Yt = oracle.residualise(Y, Q)
    coef, *_ = np.linalg.lstsq(X, Y, rcond=None)
    assert np.allclose(Yres[:, :4], (Y - X @ coef)[:, :4], atol=1e-12)
    assert np.allclose(X.T @ Yres, 0, atol=1e-10)
    assert np.allclose(np.linalg.norm(Yt[:, :4], axis=0), 1.0)
    assert np.isnan(Yt[:, 4]).all() and np.isnan(Yt[:, 5]).all()


# ---------------------------------------------------------------- OLS

def _tiny_case(seed, N=30, n_cov=2, M=7, P=3):
    r = _rng(seed)
    C = r.standard_normal((N, n_cov))
    X = oracle.design_matrix(C, N)
    g = r.integers(0, 3, size=(M, N)).astype(float)
    Y = X @ r.standard_normal((n_cov + 1, P)) + 0.3 * g[0][:, None] + r.standard_normal((N, P))
    return C, X, g, Y


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_ols_direct_vs_bruteforce_lstsq(seed):
    C, X, g, Y = _tiny_case(seed)
    beta, se, t, df = oracle.ols_direct(X, g, Y)
    N, q = X.shape
    assert df == N - q - 1
    for j in range(g.shape[0]):
        W = np.column_stack([X, g[j]])
        coef, *_ = np.linalg.lstsq(W, Y, rcond=None)
        resid = Y - W @ coef
        sigma2 = (resid ** 2).sum(0) / (N - W.shape[1])
        cov_gg = np.linalg.inv(W.T @ W)[-1, -1]
        assert np.allclose(beta[j], coef[-1], rtol=1e-10, atol=1e-12)
        assert np.allclose(se[j], np.sqrt(sigma2 * cov_gg), rtol=1e-10)
        assert np.allclose(t[j], coef[-1] / np.sqrt(sigma2 * cov_gg), rtol=1e-9)


@pytest.mark.parametrize("seed", [21, 22])
def test_direct_equals_projected_fwl(seed):
    C, X, g, Y = _tiny_case(seed, N=45, n_cov=3, M=9, P=4)
    b1, s1, t1, df1 = oracle.ols_direct(X, g, Y)
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(Y, Q)
    r, b2, s2, t2, df2, _ = oracle.ols_projected(Q, g, Yres)
    assert df1 == df2
    for a, b in ((b1, b2), (s1, s2), (t1, t2)):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-13)


def test_intercept_only_is_pearson_and_eq3():
    r = _rng(31)
    N = 50
    g = r.integers(0, 3, size=(4, N)).astype(float)
    y = r.standard_normal((N, 2)) + 0.5 * g[1][:, None]
    Q, _ = oracle.householder_basis(oracle.design_matrix(None, N))
    Yres, _, _ = oracle.residualise(y, Q)
    rr, beta, se, t, df, _ = oracle.ols_projected(Q, g, Yres)
    assert df == N - 2
    for j in range(4):
        for p in range(2):
            pear = np.corrcoef(g[j], y[:, p])[0, 1]
            assert abs(rr[j, p] - pear) < 1e-12
            assert abs(t[j, p] - pear * math.sqrt((N - 2) / (1 - pear ** 2))) < 1e-9


# ---------------------------------------------------------------- phenotypes observed on a subset

def _subset_case(seed, N=48, n_cov=2, M=5, P=3, frac=0.7):
    r = _rng(seed)
    C = r.standard_normal((N, n_cov))
    counts = r.integers(0, 3, size=(M, N)).astype(np.int8)
    miss = r.random((M, N)) < 0.15
    G = synth.pack_2bit(torch.from_numpy(counts), torch.from_numpy(miss)).numpy()
    rows = r.random(N) < frac
    Y = r.standard_normal((N, P)) + 0.4 * counts[0][:, None]
    return C, G, rows, Y


def test_subset_panel_is_ols_on_the_observed_rows_by_lstsq():
    """The test of a phenotype observed on rows S is the OLS of y_S on [1, C_S, g_S] with the
    genotype imputed by its mean over all N samples (numpy.linalg.lstsq on the subset)."""
    C, G, rows, Y = _subset_case(61)
    N = Y.shape[0]
    Ynan = Y.copy()
    Ynan[~rows] = np.nan                       # values outside S are never read
    panel = oracle.prepare_panel(Ynan, C, rows)
    assert panel["NS"] == rows.sum() and panel["df"] == rows.sum() - 3 - 1
    out = oracle.scan(G, "2bit", panel, mode="projected")
    direct = oracle.scan(G, "2bit", panel, mode="direct")
    counts, miss = oracle.decode_2bit(G, N)
    for j in range(G.shape[0]):
        obs = ~miss[j]
        g = np.where(miss[j], counts[j][obs].mean(), counts[j]).astype(float)  # all-N mean
        W = np.column_stack([np.ones(rows.sum()), C[rows], g[rows]])
        coef, *_ = np.linalg.lstsq(W, Y[rows], rcond=None)
        resid = Y[rows] - W @ coef
        df = rows.sum() - W.shape[1]
        se = np.sqrt((resid ** 2).sum(0) / df * np.linalg.inv(W.T @ W)[-1, -1])
        assert np.allclose(out["beta"][j], coef[-1], rtol=1e-9, atol=1e-12)
        assert np.allclose(out["se"][j], se, rtol=1e-9)
        assert np.allclose(direct["beta"][j], coef[-1], rtol=1e-9, atol=1e-12)
        assert np.allclose(out["t"][j], coef[-1] / se, rtol=1e-8)


def test_subset_panel_full_mask_and_outside_values():
    C, G, rows, Y = _subset_case(62)
    N = Y.shape[0]
    full = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C, np.ones(N, bool)))
    plain = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C))
    for k in ("beta", "se", "t", "mlog10p", "r"):   # equal up to BLAS summation order
        assert np.allclose(full[k], plain[k], rtol=1e-12, atol=1e-15, equal_nan=True), k
    Y2 = Y.copy()
    Y2[~rows] = 1e6 * _rng(63).standard_normal(((~rows).sum(), Y.shape[1]))
    a = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C, rows))
    b = oracle.scan(G, "2bit", oracle.prepare_panel(Y2, C, rows))
    for k in ("beta", "se", "t", "mlog10p", "r"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_subset_panel_imputation_uses_the_all_sample_mean():
    """A missing call inside S takes the marker's mean over all N observed calls: moving a
    marker's calls outside S changes the imputed value inside S, and so the statistic."""
    C, G, rows, Y = _subset_case(64, M=1)
    N = Y.shape[0]
    counts, miss = oracle.decode_2bit(G, N)
    assert (miss[0] & rows).any()
    counts2 = counts.copy()
    out_s = np.nonzero(~rows & ~miss[0])[0]
    counts2[0, out_s] = 2 - counts2[0, out_s]          # change calls outside S only
    G2 = synth.pack_2bit(torch.from_numpy(counts2.astype(np.int8)), torch.from_numpy(miss)).numpy()
    panel = oracle.prepare_panel(Y, C, rows)
    a, b = oracle.scan(G, "2bit", panel), oracle.scan(G2, "2bit", panel)
    assert counts[0][~miss[0]].mean() != counts2[0][~miss[0]].mean()
    assert not np.allclose(a["r"], b["r"])
    # the same pair with the missing calls inside S turned into observed calls of the all-N mean
    # is not expressible in codes, so check the value directly: g_S at missing calls
    g = oracle.scan(G, "2bit", panel)["decode"]["g"][0]
    assert np.allclose(g[miss[0]], counts[0][~miss[0]].mean())


def test_subset_panel_paper_form_is_pearson_on_the_subset():
    C, G, rows, Y = _subset_case(65)
    panel = oracle.prepare_panel(Y, C, rows)
    out = oracle.scan(G, "2bit", panel, mode="paper")
    assert out["df"] == rows.sum() - 2
    g = out["decode"]["g"][:, rows]
    for j in range(G.shape[0]):
        for p in range(Y.shape[1]):
            assert abs(out["r"][j, p] - np.corrcoef(g[j], panel["Yres"][:, p])[0, 1]) < 1e-12


# ---------------------------------------------------------------- the paper's printed form

def test_paper_form_is_pearson_with_residualised_phenotype():
    """Eq. 2-3 as printed: r is the Pearson correlation of the raw marker with the
    residualised phenotype (numpy.corrcoef), and the two-sided p-value is the one of a
    correlation test with N - 2 degrees of freedom (scipy.stats.pearsonr), with covariates."""
    stats = pytest.importorskip("scipy.stats")
    C, X, g, Y = _tiny_case(51, N=60, n_cov=3, M=6, P=3)
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(Y, Q)
    rr, beta, se, t, df, gc2 = oracle.ols_paper(g, Yres)
    N = X.shape[0]
    assert df == N - 2
    mlp = oracle.mlog10p_from_r(rr, df)
    for j in range(g.shape[0]):
        assert abs(gc2[j] - ((g[j] - g[j].mean()) ** 2).sum()) <= 1e-12 * gc2[j]
        for p in range(Y.shape[1]):
            pear = np.corrcoef(g[j], Yres[:, p])[0, 1]
            assert abs(rr[j, p] - pear) < 1e-12
            ref = stats.pearsonr(g[j], Yres[:, p])
            assert abs(mlp[j, p] + math.log10(ref.pvalue)) < 1e-9 * max(1.0, mlp[j, p])
            # slope of the residualised phenotype on the centred marker (numpy.polyfit)
            slope = np.polyfit(g[j] - g[j].mean(), Yres[:, p], 1)[0]
            assert abs(beta[j, p] - slope) < 1e-10 * max(1.0, abs(slope))
            assert abs(se[j, p] - abs(beta[j, p] / t[j, p])) < 1e-10 * se[j, p]


def test_paper_form_equals_ols_with_intercept_only_and_differs_with_covariates():
    """With an intercept only the printed form is the OLS test (q = 1, g_res = g_c); with
    covariates it differs by the factor |g_res| / |g_c| in r and by df."""
    C, X, g, Y = _tiny_case(52, N=50, n_cov=0, M=5, P=2)
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(Y, Q)
    a = oracle.ols_paper(g, Yres)
    b = oracle.ols_projected(Q, g, Yres)
    assert a[4] == b[4] == X.shape[0] - 2
    for x, y in zip(a[:4], b[:4]):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-14)
    C, X, g, Y = _tiny_case(53, N=50, n_cov=3, M=5, P=2)
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(Y, Q)
    rp, *_, dfp, gc2 = oracle.ols_paper(g, Yres)
    rq, *_, dfq, gres2 = oracle.ols_projected(Q, g, Yres)
    assert dfp == X.shape[0] - 2 and dfq == X.shape[0] - X.shape[1] - 1 == 45
    assert np.allclose(rp, rq * np.sqrt(gres2 / gc2)[:, None], rtol=1e-12)


def test_paper_form_scan_and_untestable_markers():
    r = _rng(54)
    N = 40
    C = r.standard_normal((N, 2))
    Y = r.standard_normal((N, 3))
    panel = oracle.prepare_panel(Y, C)
    counts = r.integers(0, 3, size=(3, N)).astype(np.int8)
    counts[0] = 1                                     # constant: untestable
    miss = np.zeros((3, N), dtype=bool)
    miss[2, :5] = True
    G = synth.pack_2bit(torch.from_numpy(counts), torch.from_numpy(miss)).numpy()
    out = oracle.scan(G, "2bit", panel, mode="paper")
    assert out["df"] == N - 2
    assert np.all(np.isnan(out["r"][0])) and np.all(np.isnan(out["mlog10p"][0]))
    assert np.all(np.isfinite(out["r"][1:]))
    g = out["decode"]["g"]
    for j in (1, 2):
        for p in range(3):
            assert abs(out["r"][j, p] - np.corrcoef(g[j], panel["Yres"][:, p])[0, 1]) < 1e-12


def test_exact_fit_gives_unit_r_and_infinite_score():
    r = _rng(41)
    N = 40
    C = r.standard_normal((N, 2))
    X = oracle.design_matrix(C, N)
    g = r.integers(0, 3, size=(1, N)).astype(float)
    y = (1.7 * g[0] + X @ np.array([0.5, -1.0, 2.0]))[:, None]
    y = np.column_stack([y, -y])
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(y, Q)
    rr, *_ , df, _ = oracle.ols_projected(Q, g, Yres)
    assert np.allclose(np.abs(rr), 1.0, atol=1e-12)
    assert rr[0, 0] > 0 > rr[0, 1]
    assert np.all(oracle.mlog10p_from_r(np.array([1.0, -1.0]), df) == np.inf)


def test_untestable_markers_are_nan():
    r = _rng(42)
    N = 30
    C = r.standard_normal((N, 2))
    X = oracle.design_matrix(C, N)
    g = np.vstack([np.full(N, 1.0), 2.0 * C[:, 0] + 1.0, r.integers(0, 3, N)])
    Y = r.standard_normal((N, 2))
    Q, _ = oracle.householder_basis(X)
    Yres, _, _ = oracle.residualise(Y, Q)
    rr, b, s, t, df, gres2 = oracle.ols_projected(Q, g, Yres)
    assert np.isnan(rr[:2]).all() and np.isfinite(rr[2]).all()
    b1, s1, t1, _ = oracle.ols_direct(X, g, Y)
    assert np.isnan(b1[:2]).all() and np.isfinite(b1[2]).all()


def _marker_with_vif(seed, N, vif, n_other=2):
    """A 0/1/2 marker g and covariates C such that g's variance inflation factor on [1, C] is
    `vif` by construction: C[:, 0] = g_c + lam e with e orthogonal to 1 and g_c, so that the
    residual of g_c on [1, C[:, 0]] has |g_res|^2 / |g_c|^2 = lam^2 |e|^2 / (|g_c|^2 + lam^2 |e|^2)
    = 1 / vif; the other covariates are orthogonal to 1, g_c and e, so they change nothing."""
    r = _rng(seed)
    g = r.integers(0, 3, N).astype(float)
    gc = g - g.mean()
    B = np.column_stack([np.ones(N), gc])
    e = r.standard_normal(N)
    e -= B @ np.linalg.lstsq(B, e, rcond=None)[0]
    rho = 1.0 / vif
    lam = math.sqrt((gc @ gc) * rho / (1.0 - rho) / (e @ e))
    O = r.standard_normal((N, n_other))
    B3 = np.column_stack([B, e])
    O -= B3 @ np.linalg.lstsq(B3, O, rcond=None)[0]
    C = np.column_stack([gc + lam * e, O])
    return g, C


@pytest.mark.parametrize("N", [60, 400])
def test_marker_cut_either_side_of_the_variance_inflation_limit(N):
    """Markers built at VIF = 50 (1 -/+ 1e-6), and far from the limit (VIF 10 and 1,000): the
    direct OLS and the projected form test the ones at or below 50 and give NaN above it. The
    VIF of each construction is checked independently (R^2 of g on [1, C] by lstsq)."""
    cases = [(50.0 * (1 - 1e-6), True), (50.0 * (1 + 1e-6), False), (10.0, True), (1000.0, False)]
    for k, (vif, tested) in enumerate(cases):
        g, C = _marker_with_vif(100 + k, N, vif)
        X = oracle.design_matrix(C, N)
        coef, *_ = np.linalg.lstsq(X, g, rcond=None)
        res = g - X @ coef
        gc = g - g.mean()
        assert abs((gc @ gc) / (res @ res) / vif - 1.0) < 1e-9
        Y = X @ _rng(k).standard_normal((X.shape[1], 2)) + 0.5 * g[:, None] + _rng(200 + k).standard_normal((N, 2))
        beta, se, t, df = oracle.ols_direct(X, g[None, :], Y)
        Q, _ = oracle.householder_basis(X)
        Yres, _, _ = oracle.residualise(Y, Q)
        rr, b2, s2, t2, _, gres2 = oracle.ols_projected(Q, g[None, :], Yres)
        assert bool(np.isfinite(beta).all()) == tested and bool(np.isnan(beta).all()) == (not tested), vif
        assert bool(np.isfinite(rr).all()) == tested and bool(np.isnan(rr).all()) == (not tested), vif
        if tested:  # the values next to the limit are the OLS ones (brute force)
            W = np.column_stack([X, g])
            cw, *_ = np.linalg.lstsq(W, Y, rcond=None)
            assert np.allclose(beta[0], cw[-1], rtol=1e-8)
            assert np.allclose(b2[0], cw[-1], rtol=1e-8)
            assert abs(gres2[0] / (res @ res) - 1.0) < 1e-9


def test_testable_rule_at_the_limit():
    """The rule itself: tested iff |g_c|^2 > 0 and |g_c|^2 / |g_res|^2 <= 50."""
    from oracle.ols import MAX_VIF, testable
    assert MAX_VIF == 50.0
    gc2 = np.array([50.0, 50.0, 50.0, 0.0, 1.0, np.nan])
    gres2 = np.array([1.0, 1.0 - 1e-12, 1.0 + 1e-12, 0.0, 1.0, 1.0])
    assert testable(gc2, gres2).tolist() == [True, False, True, False, True, False]


# ---------------------------------------------------------------- p-values

def _p_df1(t):
    return (2 / math.pi) * math.atan(1 / abs(t)) if t != 0 else 1.0


def _p_df2(t):
    s = math.sqrt(2 + t * t)
    return 2 / (s * (s + abs(t)))


def _p_df3(t):
    u = abs(t) / math.sqrt(3)
    if u == 0:
        return 1.0
    return (2 / math.pi) * (math.atan(1 / u) - u / (1 + u * u)) if u < 1 else \
        1 - (2 / math.pi) * (math.atan(u) + u / (1 + u * u))


@pytest.mark.parametrize("df,fn", [(1, _p_df1), (2, _p_df2), (3, _p_df3)])
def test_pvalue_closed_forms(df, fn):
    ts = [0.0, 1e-6, 0.3, 1.0, 2.5, 7.0, 40.0, 1e3, 1e6]
    got = oracle.mlog10p_from_t(np.array(ts), df)
    for t, v in zip(ts, got):
        if df == 3 and abs(t) / math.sqrt(3) >= 1 and t > 10:
            continue   # the df=3 closed form loses accuracy to cancellation there
        exp = -math.log10(fn(t))
        assert abs(v - exp) <= 1e-10 * max(1.0, abs(exp)), (t, v, exp)


def test_pvalue_df1_df2_extreme_tail_log_space():
    # p far below the float64 range of 1 - I: only a log-space evaluation gets these
    t = np.array([1e20, 1e100])
    exp1 = [-math.log10(2 / math.pi) + math.log10(x) for x in t]          # p ~ 2/(pi t)
    got1 = oracle.mlog10p_from_t(t, 1)
    assert np.allclose(got1, exp1, rtol=1e-12)
    exp2 = [-math.log10(1.0) + 2 * math.log10(x) for x in t]              # p ~ 1/t^2
    got2 = oracle.mlog10p_from_t(t, 2)
    assert np.allclose(got2, exp2, rtol=1e-12)


def test_pvalue_published_t_table():
    for line in open(os.path.join(GOLDEN, "t_table_two_sided.txt")):
        if line.startswith("#") or not line.strip():
            continue
        d, alpha, tc = line.split()
        df = 1e12 if d == "inf" else float(d)
        alpha, tc = float(alpha), float(tc)
        lo, hi = (10 ** -oracle.mlog10p_from_t(np.array([tc + 5e-4, tc - 5e-4]), df))
        assert lo <= alpha <= hi, (d, alpha, tc, lo, hi)


def test_pvalue_normal_limit():
    # t with df = 1e8 differs from the normal tail by a relative O(z^4 / df) in p
    z = np.array([0.5, 1.96, 4.0, 8.0])
    got = oracle.mlog10p_from_t(z, 1e8)
    exp = np.array([-math.log10(math.erfc(v / math.sqrt(2))) for v in z])
    assert np.allclose(got, exp, rtol=1e-6)


def test_pvalue_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for df in (7.0, 1995.0, 22979.0):
        for t in (0.01, 0.8, 3.3, 6.0, 12.0, 21.7, 60.0):
            x = mp.mpf(df) / (df + mp.mpf(t) ** 2)
            p = mp.betainc(df / 2, mp.mpf(1) / 2, 0, x, regularized=True)
            exp = float(-mp.log10(p))
            got = float(oracle.mlog10p_from_t(np.array([t]), df)[0])
            assert abs(got - exp) <= 1e-11 * max(1.0, exp), (df, t, got, exp)


def test_pvalue_from_r_matches_from_t():
    r = np.array([0.0, 1e-4, 0.02, 0.14, 0.5, 0.9, 0.999999])
    df = 22979
    t = r * np.sqrt(df / ((1 - r) * (1 + r)))
    assert np.allclose(oracle.mlog10p_from_r(r, df), oracle.mlog10p_from_t(t, df), rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------- invariances

def _panel_case(seed, N=120, n_cov=3, M=12, P=5):
    r = _rng(seed)
    C = r.standard_normal((N, n_cov))
    counts = r.integers(0, 3, size=(M, N))
    miss = r.random((M, N)) < 0.05
    G = synth.pack_2bit(torch.from_numpy(counts.astype(np.int8)), torch.from_numpy(miss)).numpy()
    Y = r.standard_normal((N, P)) + C @ r.standard_normal((n_cov, P)) + 0.4 * counts[2][:, None]
    return C, counts, miss, G, Y


def test_invariance_sample_permutation():
    C, counts, miss, G, Y = _panel_case(51)
    N = Y.shape[0]
    perm = _rng(52).permutation(N)
    a = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C))
    Gp = synth.pack_2bit(torch.from_numpy(counts[:, perm].astype(np.int8)),
                         torch.from_numpy(miss[:, perm])).numpy()
    b = oracle.scan(Gp, "2bit", oracle.prepare_panel(Y[perm], C[perm]))
    for k in ("beta", "se", "t", "mlog10p"):
        assert np.allclose(a[k], b[k], rtol=1e-9, atol=1e-12)


def test_invariance_phenotype_affine_and_allele_flip():
    C, counts, miss, G, Y = _panel_case(53)
    N = Y.shape[0]
    X = oracle.design_matrix(C, N)
    a = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C))
    Y2 = -2.5 * Y + X @ _rng(54).standard_normal((X.shape[1], Y.shape[1]))
    b = oracle.scan(G, "2bit", oracle.prepare_panel(Y2, C))
    assert np.allclose(b["beta"], -2.5 * a["beta"], rtol=1e-9)
    assert np.allclose(b["t"], -a["t"], rtol=1e-9)
    assert np.allclose(b["mlog10p"], a["mlog10p"], rtol=1e-9)
    flip = synth.pack_2bit(torch.from_numpy((2 - counts).astype(np.int8)), torch.from_numpy(miss)).numpy()
    c = oracle.scan(flip, "2bit", oracle.prepare_panel(Y, C))
    assert np.allclose(c["beta"], -a["beta"], rtol=1e-9)
    assert np.allclose(c["mlog10p"], a["mlog10p"], rtol=1e-9)


def test_invariance_redundant_covariate():
    C, counts, miss, G, Y = _panel_case(55)
    a = oracle.scan(G, "2bit", oracle.prepare_panel(Y, C))
    C2 = np.column_stack([C, C[:, 0] - 2 * C[:, 2], np.ones(C.shape[0])])
    pan = oracle.prepare_panel(Y, C2)
    assert pan["q"] == C.shape[1] + 1
    b = oracle.scan(G, "2bit", pan)
    for k in ("beta", "se", "t", "mlog10p"):
        assert np.allclose(a[k], b[k], rtol=1e-9, atol=1e-12)


def test_direct_and_projected_scan_agree_with_missing_calls():
    C, counts, miss, G, Y = _panel_case(56)
    pan = oracle.prepare_panel(Y, C)
    a = oracle.scan(G, "2bit", pan, mode="direct")
    b = oracle.scan(G, "2bit", pan, mode="projected")
    for k in ("beta", "se", "t", "mlog10p"):
        assert np.allclose(a[k], b[k], rtol=1e-9, atol=1e-12), k


# ---------------------------------------------------------------- ranking

def test_hits_and_best():
    mlp = np.array([[1.0, 9.0, np.nan], [8.0, 2.0, 3.0], [8.0, np.nan, 7.5]])
    h = oracle.hits(mlp, 7.5, marker_offset=100)
    assert h.tolist() == [[100, 1], [101, 0], [102, 0], [102, 2]]
    r = np.array([[0.1, -0.5, np.nan], [0.3, 0.5, np.nan], [-0.3, 0.2, np.nan]])
    assert oracle.best_per_phenotype(r).tolist() == [1, 0, -1]


def test_planted_loci_rank_top_small_workload():
    w = synth.WORKLOADS["n2000_m10000_p16_c5_2bit"]
    pan_in = synth.make_panel(w)
    blk = synth.make_block(w, 0)
    Y = pan_in["Yt"].numpy().T.astype(np.float64)
    C = pan_in["cov_t"].numpy().T
    pan = oracle.prepare_panel(Y, C)
    res = oracle.scan(blk["G"].numpy(), "2bit", pan)
    found = 0
    for m, p in pan_in["pairs"]:
        top = np.argsort(-np.abs(res["r"][:, p]))[: w.causal_per_pheno]
        found += m in top
    assert found >= 0.9 * len(pan_in["pairs"])
    assert res["df"] == w.N - (w.n_cov + 1) - 1


def test_large_df_normal_deviate_used_on_gpu_is_within_tolerance():
    """The GPU evaluates -log10 p of FULL elements for df >= 1500 from Hill's (1970) normal
    deviate for Student's t instead of the continued fraction (which cancels badly in FP32 at
    large df); elements with 1 - r^2 < 0.05 (t > sqrt(19 df)) and every hit take the FP64
    continued fraction instead. This pins the approximation itself, evaluated here in float64,
    against the oracle over every t it is used on, t in [0.01, max(400, sqrt(19 df))], for df
    up to 1e7 (t up to 1.4e4)."""
    sp = pytest.importorskip("scipy.special")

    def hill_mlog10p(t, n):
        a = n - 0.5
        B = 48 * a * a
        Y = a * math.log1p(t * t / n)
        z = (((((-0.4 * Y - 3.3) * Y - 24) * Y - 85.5) / (0.8 * Y * Y + 100 + B) + Y + 3) / B + 1) * math.sqrt(Y)
        x = z / math.sqrt(2)
        return (x * x - math.log(sp.erfcx(x))) / math.log(10)

    for n in (1500.0, 1994.0, 5000.0, 22979.0, 1e5, 1e6, 1e7):
        tmax = max(400.0, math.sqrt(19.0 * n))
        ts = np.concatenate([np.linspace(0.01, 10, 200), np.geomspace(10, tmax, 120)])
        ref = oracle.mlog10p_from_t(ts, n)
        got = np.array([hill_mlog10p(t, n) for t in ts])
        assert np.all(np.abs(got - ref) <= 0.1 * np.maximum(1e-3, 1e-5 * ref)), n
