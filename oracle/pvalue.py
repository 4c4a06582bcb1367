"""Two-sided Student-t p-values in log space (Section 2.2: t "converted directly to P values").

Test infrastructure (see the package docstring).

For a t statistic with df degrees of freedom the two-sided p-value is the
regularised incomplete beta function p = I_x(df/2, 1/2) with x = df / (df + t^2);
for a correlation r, x = 1 - r^2 (Eq. 3 makes df/(df + t^2) = 1 - r^2).

I_x(a, b) is evaluated from its continued fraction (Abramowitz & Stegun 26.5.8)
with the modified Lentz method (Lentz 1976; Thompson & Barnett 1986), in log space
so that no p-value underflows, and through the symmetry I_x(a, b) = 1 - I_{1-x}(b, a)
when x >= (a + 1) / (a + b + 2), where the fraction converges slowly. x and 1 - x are
always passed separately so that neither is formed by cancellation.
"""
from __future__ import annotations

import math

import numpy as np

_TINY = 1e-300
_EPS = 1e-16
_MAX_ITER = 100_000
_LN10 = math.log(10.0)


def _lentz_cf(a: float, b: float, x: np.ndarray) -> np.ndarray:
    """Value h of the continued fraction with I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * h."""
    x = np.asarray(x, dtype=np.float64)
    h = np.empty_like(x)
    idx = np.arange(x.size)
    xs = x.ravel().copy()
    c = np.ones_like(xs)
    d = 1.0 - (a + b) * xs / (a + 1.0)
    d = np.where(np.abs(d) < _TINY, _TINY, d)
    d = 1.0 / d
    hh = d.copy()
    out = h.ravel()
    for m in range(1, _MAX_ITER + 1):
        for num in (m * (b - m) * xs / ((a + 2 * m - 1.0) * (a + 2 * m)),
                    -(a + m) * (a + b + m) * xs / ((a + 2 * m) * (a + 2 * m + 1.0))):
            d = 1.0 + num * d
            d = np.where(np.abs(d) < _TINY, _TINY, d)
            c = 1.0 + num / c
            c = np.where(np.abs(c) < _TINY, _TINY, c)
            d = 1.0 / d
            step = d * c
            hh = hh * step
        done = np.abs(step - 1.0) <= _EPS
        if done.any():
            out[idx[done]] = hh[done]
            keep = ~done
            idx, xs, c, d, hh = idx[keep], xs[keep], c[keep], d[keep], hh[keep]
            if idx.size == 0:
                return out.reshape(x.shape)
    raise RuntimeError("incomplete beta continued fraction did not converge")


def log_betainc(a: float, b: float, lnx: np.ndarray, lny: np.ndarray) -> np.ndarray:
    """ln I_x(a, b) given ln x and ln(1 - x) (arrays of the same shape)."""
    lnx = np.asarray(lnx, dtype=np.float64)
    lny = np.asarray(lny, dtype=np.float64)
    x = np.exp(lnx)
    y = np.exp(lny)
    lnB = math.lgamma(a) + math.lgamma(b) - math.lgamma(a + b)
    out = np.full(x.shape, np.nan)
    direct = x < (a + 1.0) / (a + b + 2.0)
    fin = np.isfinite(lnx) & np.isfinite(lny)
    out[(lnx == -np.inf) & ~np.isnan(lny)] = -np.inf     # x = 0: I = 0
    out[(lny == -np.inf) & ~np.isnan(lnx)] = 0.0         # x = 1: I = 1
    sel = fin & direct
    if sel.any():
        h = _lentz_cf(a, b, x[sel])
        out[sel] = a * lnx[sel] + b * lny[sel] - math.log(a) - lnB + np.log(h)
    sel = fin & ~direct
    if sel.any():
        h = _lentz_cf(b, a, y[sel])
        comp = np.exp(b * lny[sel] + a * lnx[sel] - math.log(b) - lnB + np.log(h))
        with np.errstate(divide="ignore"):
            out[sel] = np.log1p(-np.minimum(comp, 1.0))
    return out


def _mlog10p(lnx: np.ndarray, lny: np.ndarray, df) -> np.ndarray:
    df = np.broadcast_to(np.asarray(df, dtype=np.float64), np.shape(lnx))
    out = np.full(np.shape(lnx), np.nan)
    for d in np.unique(df[np.isfinite(df)]):
        sel = df == d
        out[sel] = -log_betainc(0.5 * d, 0.5, lnx[sel], lny[sel]) / _LN10
    return out


def mlog10p_from_t(t, df) -> np.ndarray:
    """-log10 of the two-sided p-value of Student's t with df degrees of freedom."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    df = np.asarray(df, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        lu = 2.0 * np.log(t) - np.log(df)             # ln(t^2 / df), no overflow
        big = lu > 0
        e = np.exp(np.where(big, -lu, lu))            # u or 1/u, whichever is <= 1
        l1 = np.log1p(e)
        lnx = np.where(big, -(lu + l1), -l1)          # ln(df / (df + t^2)) = -ln(1 + u)
        lny = np.where(big, -l1, lu - l1)             # ln(t^2 / (df + t^2)) = ln u - ln(1 + u)
    lnx = np.where(np.isinf(t), -np.inf, lnx)
    lny = np.where(np.isinf(t), 0.0, lny)
    lnx = np.where(np.isnan(t), np.nan, lnx)
    lny = np.where(np.isnan(t), np.nan, lny)
    return _mlog10p(np.atleast_1d(lnx), np.atleast_1d(lny), df).reshape(t.shape)


def mlog10p_from_r(r, df) -> np.ndarray:
    """-log10 p of the correlation test with df degrees of freedom (x = 1 - r^2, 1 - x = r^2)."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        lnx = np.log((1.0 - a) * (1.0 + a))
        lny = 2.0 * np.log(a)
    return _mlog10p(np.atleast_1d(lnx), np.atleast_1d(lny), df).reshape(a.shape)
