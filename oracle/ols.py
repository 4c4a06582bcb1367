"""Per-marker least squares: the linear association test the scan computes (Section 2.2).

Test infrastructure (see the package docstring).

The paper states its test as a correlation of standardised genotypes with the
residualised, standardised panel (Eq. 2) turned into t (Eq. 3), "equivalent to a
correlation-based linear association test". The test it stands for is the OLS fit
of each phenotype on [1, C, g] per marker; `ols_direct` solves exactly that, and
`ols_projected` computes the same numbers the way Eq. 1-3 do (project, correlate,
convert), with the genotype projected on Q as well (Frisch-Waugh-Lovell).

Reading: degrees of freedom df = N - q - 1 (q = rank [1, C]); with an intercept
only, q = 1 and df = N - 2 as in Eq. 3.

`ols_paper` is the statistic exactly as Section 2.2 prints it: the marker is only centred
and standardised (not projected on Q), r is its correlation with the residualised panel,
and Eq. 3 uses N - 2 degrees of freedom whatever the covariates. It equals the OLS test
when the covariates are an intercept only.
"""
from __future__ import annotations

import numpy as np

# Reading (the paper is silent on collinear markers): a marker is untestable when it has no
# observed call, is constant, or its variance inflation factor on the covariates,
#   VIF = |g_c|^2 / |g_res|^2 = 1 / (1 - R^2 of g on [1, C]),
# exceeds MAX_VIF = 50, i.e. the covariates explain more than 98% of its variance. The sampling
# variance of the marker's effect is inflated by exactly this factor; 50 is the limit that
# PLINK's linear model applies by default to each of its predictors (PLINK is the tool the
# paper checks its concordance against, Section 3.1). A marker exactly at the limit is tested.
MAX_VIF = 50.0


def testable(gc2, gres2):
    """True where a marker with |g_c|^2 = gc2 and |g_res|^2 = gres2 is tested (NaN: not)."""
    gc2 = np.asarray(gc2, dtype=np.float64)
    gres2 = np.asarray(gres2, dtype=np.float64)
    return (gc2 > 0.0) & (MAX_VIF * gres2 >= gc2)


def ols_direct(X: np.ndarray, g: np.ndarray, Y: np.ndarray):
    """OLS of every column of Y on W = [X, g_j] for each marker j, by QR of W.

    X: [N][q] full column rank; g: [M][N] imputed genotypes; Y: [N][P].
    Returns (beta, se, t) each [M][P] (the coefficient of g_j, its standard error
    sqrt(RSS/df * [(W^T W)^-1]_gg), and beta/se) and df. Untestable markers give NaN.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    N, q = X.shape
    M, P = g.shape[0], Y.shape[1]
    df = N - q - 1
    beta = np.full((M, P), np.nan)
    se = np.full((M, P), np.nan)
    for j in range(M):
        if not np.all(np.isfinite(g[j])):
            continue
        W = np.column_stack([X, g[j]])
        Qw, Rw = np.linalg.qr(W)
        gc = g[j] - g[j].mean()
        rgg = abs(Rw[-1, -1])                 # |g_res|: what is left of g after [1, C]
        if not np.isfinite(rgg) or not testable(gc @ gc, rgg * rgg):
            continue
        coef = np.linalg.solve(Rw, Qw.T @ Y)
        resid = Y - W @ coef
        rss = (resid * resid).sum(axis=0)
        beta[j] = coef[-1]
        se[j] = np.sqrt(rss / df) / rgg
    with np.errstate(invalid="ignore", divide="ignore"):
        t = beta / se
    return beta, se, t, df


def ols_projected(Q: np.ndarray, g: np.ndarray, Yres: np.ndarray):
    """Eq. 2 and Eq. 3 with the genotype projected on Q too (FWL form of the same OLS).

    Q: [N][q] orthonormal basis of [1, C]; g: [M][N] imputed genotypes; Yres: [N][P]
    residualised panel (Eq. 1). r = g_res . y_res / (|g_res| |y_res|),
    t = r sqrt(df / (1 - r^2)), beta = g_res . y_res / |g_res|^2, se = |beta / t|.
    Returns (r, beta, se, t, df, gres2 [M] = |g_res|^2).
    """
    Q = np.asarray(Q, dtype=np.float64)
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    Yres = np.asarray(Yres, dtype=np.float64)
    N, q = Q.shape
    df = N - q - 1
    gc = g - g.mean(axis=1, keepdims=True)
    gres = gc - (gc @ Q) @ Q.T
    gres2 = (gres * gres).sum(axis=1)
    gc2 = (gc * gc).sum(axis=1)
    bad = ~testable(gc2, gres2)
    ynorm = np.linalg.norm(Yres, axis=0)
    num = gres @ Yres
    with np.errstate(invalid="ignore", divide="ignore"):
        r = num / np.sqrt(gres2)[:, None] / ynorm[None, :]
        r = np.clip(r, -1.0, 1.0)
        t = r * np.sqrt(df / ((1.0 - r) * (1.0 + r)))
        beta = num / gres2[:, None]
        se = ynorm[None, :] * np.sqrt((1.0 - r) * (1.0 + r) / df) / np.sqrt(gres2)[:, None]
    for a in (r, beta, se, t):
        a[bad] = np.nan
    return r, beta, se, t, df, np.where(bad, np.nan, gres2)


def ols_paper(g: np.ndarray, Yres: np.ndarray):
    """Eq. 2 and Eq. 3 as printed in Section 2.2 (the genotype is not projected on Q).

    g: [M][N] imputed genotypes; Yres: [N][P] residualised panel (Eq. 1).
    r = g_c . y_res / (|g_c| |y_res|) with g_c = g - mean(g) (the standardised marker),
    t = r sqrt((N - 2) / (1 - r^2)) (Eq. 3), df = N - 2.
    Reading (the paper reports no effect size): beta = g_c . y_res / |g_c|^2, the slope of
    the residualised phenotype on the centred marker, and se = |beta / t|.
    A marker with no observed call or a constant one is untestable (NaN).
    Returns (r, beta, se, t, df, gc2 [M] = |g_c|^2).
    """
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    Yres = np.asarray(Yres, dtype=np.float64)
    N = g.shape[1]
    df = N - 2
    gc = g - g.mean(axis=1, keepdims=True)
    gc2 = (gc * gc).sum(axis=1)
    bad = ~(gc2 > 0.0)
    ynorm = np.linalg.norm(Yres, axis=0)
    num = gc @ Yres
    with np.errstate(invalid="ignore", divide="ignore"):
        r = num / np.sqrt(gc2)[:, None] / ynorm[None, :]
        r = np.clip(r, -1.0, 1.0)
        t = r * np.sqrt(df / ((1.0 - r) * (1.0 + r)))
        beta = num / gc2[:, None]
        se = ynorm[None, :] * np.sqrt((1.0 - r) * (1.0 + r) / df) / np.sqrt(gc2)[:, None]
    for a in (r, beta, se, t):
        a[bad] = np.nan
    return r, beta, se, t, df, np.where(bad, np.nan, gc2)
