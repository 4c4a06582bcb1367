"""Covariate basis and panel residualisation (Section 2.2, Eq. 1 and the standardisation after it).

Test infrastructure (see the package docstring).

Readings taken where the paper is silent:

* Q spans the design [1, C]: the intercept is always included, so the centring of
  Eq. 1 is part of the projection, and a covariate that is already in the span of
  the columns before it is dropped (rank detection). q = rank([1, C]).
* Rank rule: a column is dropped when the norm of what is left of it after the
  reflections of the kept columns before it is at most 1e-9 times its own norm.
* Standardisation to unit variance is taken as unit Euclidean norm; the paper's
  /N in Eq. 2 then cancels (correlations are unchanged by a common scale).
* A phenotype whose residual norm is at most 1e-12 times the norm of the centred
  phenotype (constant, or inside the covariate span) has no test: its column is NaN.
"""
from __future__ import annotations

import numpy as np

RANK_TOL = 1e-9
PHENO_TOL = 1e-12


def design_matrix(C: np.ndarray | None, N: int) -> np.ndarray:
    """X = [1, C]: float64 [N][1 + n_cov]; C is [N][n_cov] (or None)."""
    ones = np.ones((N, 1))
    if C is None or np.size(C) == 0:
        return ones
    return np.hstack([ones, np.asarray(C, dtype=np.float64).reshape(N, -1)])


def householder_basis(X: np.ndarray, tol: float = RANK_TOL):
    """Orthonormal basis of span(X) by Householder reflections with column dropping.

    Returns (Q float64 [N][q], kept column indices). Q's columns are H_0 ... H_{q-1}
    applied to the first q unit vectors, so Q[:, k] spans the k-th kept column
    after removing the kept columns before it.
    """
    X = np.array(X, dtype=np.float64)
    N, k = X.shape
    R = X.copy()
    refl = []
    kept = []
    row = 0
    for j in range(k):
        if row >= N:
            break
        own = np.linalg.norm(X[:, j])
        x = R[row:, j]
        nrm = np.linalg.norm(x)
        if own == 0.0 or nrm <= tol * own:
            continue
        v = x.copy()
        v[0] += nrm if x[0] >= 0 else -nrm
        v /= np.linalg.norm(v)
        R[row:, :] -= 2.0 * np.outer(v, v @ R[row:, :])
        refl.append((row, v))
        kept.append(j)
        row += 1
    q = row
    Q = np.zeros((N, q))
    Q[:q, :q] = np.eye(q)
    for r, v in reversed(refl):
        Q[r:, :] -= 2.0 * np.outer(v, v @ Q[r:, :])
    return Q, kept


def residualise(Y: np.ndarray, Q: np.ndarray):
    """Eq. 1: Y_res = (I - Q Q^T)(Y - Ybar), then unit-norm columns.

    Y: float64 [N][P]. Returns (Y_res [N][P], s [P] = column norms of Y_res,
    Ytilde [N][P] = Y_res / s; a column without a test gives NaN).
    """
    Y = np.asarray(Y, dtype=np.float64)
    Yc = Y - Y.mean(axis=0, keepdims=True)
    Yres = Yc - Q @ (Q.T @ Yc)
    s = np.linalg.norm(Yres, axis=0)
    ok = s > PHENO_TOL * np.linalg.norm(Yc, axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        Yt = Yres / np.where(ok, s, np.nan)
    return Yres, s, Yt
