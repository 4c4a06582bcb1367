"""The whole genome scan in FP64 (Section 2.1 design, Section 2.2 Eq. 1-3).

Test infrastructure (see the package docstring).

`prepare_panel` builds Q and the residualised, standardised panel once (Section 2.1:
the panel is residualised and standardised once and reused); `scan` tests every
marker of a genotype block against every phenotype, either by direct OLS (the
definition) or by the projected form of Eq. 1-3; `hits` and `best_per_phenotype`
give the ranking the paper mentions after Eq. 3.

Readings: hits are the (marker, phenotype) pairs with -log10 p >= threshold,
listed by marker then phenotype; the best marker of a phenotype is the one with the
largest |r| (equivalently |t|), ties going to the smaller marker index.
"""
from __future__ import annotations

import numpy as np

from .decode import DOSAGE_SCALE, decode_2bit, decode_u8, impute, marker_stats
from .ols import ols_direct, ols_paper, ols_projected
from .panel import design_matrix, householder_basis, residualise
from .pvalue import mlog10p_from_r, mlog10p_from_t


def prepare_panel(Y: np.ndarray, C: np.ndarray | None, samples: np.ndarray | None = None) -> dict:
    """Y: [N][P] phenotypes; C: [N][n_cov] covariates (intercept not included).

    samples: optional bool [N], the samples these phenotypes are observed on (a group of
    phenotypes sharing one missingness pattern). Reading (the paper has no missing
    phenotypes): the panel is then Eq. 1 and the standardisation applied to those rows only,
    X = [1, C] restricted to them, and every test below uses only those rows (df = N_S - q - 1);
    phenotype values outside them are never read. Genotype imputation stays a property of the
    marker: a missing call is imputed with the marker's mean over all N samples.
    """
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.shape[0]
    rows = None if samples is None else np.asarray(samples, dtype=bool)
    if rows is not None:
        assert rows.shape == (N,)
        Y = Y[rows]
        C = None if C is None or np.size(C) == 0 else np.asarray(C, dtype=np.float64).reshape(N, -1)[rows]
    NS = Y.shape[0]
    X = design_matrix(C, NS)
    Q, kept = householder_basis(X)
    Yres, s, Yt = residualise(Y, Q)
    q = Q.shape[1]
    return {"N": N, "NS": NS, "rows": rows, "P": Y.shape[1], "X": X, "Xk": X[:, kept],
            "kept": kept, "Q": Q, "q": q, "df": NS - q - 1, "Y": Y, "Yres": Yres, "s": s,
            "Yt": Yt, "pheno_ok": np.isfinite(Yt).all(axis=0)}


def decode(G: np.ndarray, encoding: str, N: int, missing_words=None) -> dict:
    if encoding == "2bit":
        assert missing_words is None
        units, miss = decode_2bit(G, N)
        scale = 1.0
    elif encoding == "u8":
        units, miss = decode_u8(G, N, missing_words)
        scale = DOSAGE_SCALE
    else:
        raise ValueError(encoding)
    n_obs, S, S2, mean_units = marker_stats(units, miss)
    g = impute(units, miss, mean_units, scale)
    return {"units": units, "missing": miss, "n_obs": n_obs, "S": S, "S2": S2,
            "mean_units": mean_units, "scale": scale, "g": g}


def scan(G: np.ndarray, encoding: str, panel: dict, missing_words=None, mode: str = "projected") -> dict:
    """Statistics of every (marker, phenotype) pair of one genotype block.

    Modes: "direct" (OLS of y on [1, C, g], the definition), "projected" (Eq. 1-3 with the
    marker projected on Q as well; the same numbers) and "paper" (Eq. 2-3 exactly as
    printed: the marker only standardised, df = N - 2).
    Returns beta, se, t, mlog10p ([M][P]; r too in projected and paper mode), df, the decode
    record and gres2 (|g_res|^2 per marker in allele units; |g_c|^2 in paper mode).
    """
    dec = decode(G, encoding, panel["N"], missing_words)
    g = dec["g"]                       # imputed over all N samples
    if panel.get("rows") is not None:  # a panel of a sample subset tests those rows only
        g = g[:, panel["rows"]]
    ok = panel["pheno_ok"]
    out = {"df": panel["df"], "decode": dec}
    if mode == "direct":
        beta, se, t, df = ols_direct(panel["Xk"], g, panel["Y"])
        mlp = mlog10p_from_t(t, df)
    elif mode == "projected":
        r, beta, se, t, df, gres2 = ols_projected(panel["Q"], g, panel["Yres"])
        mlp = mlog10p_from_r(r, df)
        r[:, ~ok] = np.nan
        out["r"] = r
        out["gres2"] = gres2
    elif mode == "paper":
        r, beta, se, t, df, gc2 = ols_paper(g, panel["Yres"])
        mlp = mlog10p_from_r(r, df)
        r[:, ~ok] = np.nan
        out["r"] = r
        out["gres2"] = gc2
        out["df"] = df
    else:
        raise ValueError(mode)
    for a in (beta, se, t, mlp):
        a[:, ~ok] = np.nan
    out.update(beta=beta, se=se, t=t, mlog10p=mlp)
    return out


def hits(mlog10p: np.ndarray, threshold: float, marker_offset: int = 0) -> np.ndarray:
    """(marker, phenotype) pairs with -log10 p >= threshold, sorted; int64 [H][2]."""
    j, p = np.nonzero(np.nan_to_num(mlog10p, nan=-np.inf) >= threshold)
    order = np.lexsort((p, j))
    return np.stack([j[order] + marker_offset, p[order]], axis=1)


def best_per_phenotype(stat: np.ndarray) -> np.ndarray:
    """Per phenotype, the marker with the largest |stat| (smallest index on ties); -1 if none."""
    a = np.abs(np.asarray(stat, dtype=np.float64))
    a = np.where(np.isnan(a), -np.inf, a)
    best = np.argmax(a, axis=0)
    best[~np.isfinite(a.max(axis=0)) & (a.max(axis=0) == -np.inf)] = -1
    return best
