"""Genotype decoding and mean imputation (Section 2.2: genotypes processed in batches of markers).

Test infrastructure (see the package docstring).

The paper reads PLINK and BGEN inputs (Abstract; Section 1) without giving an
encoding. Readings taken here:

* 2-bit calls follow the PLINK 1 .bed SNP-major layout: sample i sits in bits
  2(i%4)..2(i%4)+1 of byte i//4 of the marker's row, and the field counts allele 1:
  0b00 -> 2, 0b10 -> 1, 0b11 -> 0, 0b01 -> missing.
* 8-bit dosages: byte b is the allele-1 dosage 2b/255; missing calls come only
  from a separate bit mask (bit i%32 of 32-bit word i//32 set = missing).
* A missing call is imputed with the marker's observed mean.
"""
from __future__ import annotations

import numpy as np

_BED_FIELD_TO_COUNT = {0b00: 2, 0b10: 1, 0b11: 0}
_BED_MISSING = 0b01

DOSAGE_SCALE = 2.0 / 255.0


def decode_2bit(G: np.ndarray, N: int):
    """G: uint8 [M][ldg] packed rows. Returns (counts int64 [M][N], missing bool [M][N]);
    counts are 0 under a missing call."""
    G = np.asarray(G, dtype=np.uint8)
    M = G.shape[0]
    counts = np.zeros((M, N), dtype=np.int64)
    missing = np.zeros((M, N), dtype=bool)
    for i in range(N):
        field = (G[:, i // 4].astype(np.int64) >> (2 * (i % 4))) & 0b11
        missing[:, i] = field == _BED_MISSING
        for f, c in _BED_FIELD_TO_COUNT.items():
            counts[field == f, i] = c
    return counts, missing


def unpack_mask(words: np.ndarray | None, M: int, N: int) -> np.ndarray:
    """Bit-packed missing mask int32 [M][ceil(N/32)] -> bool [M][N]."""
    if words is None:
        return np.zeros((M, N), dtype=bool)
    w = np.asarray(words).astype(np.int64) & 0xFFFFFFFF
    i = np.arange(N)
    return ((w[:, i // 32] >> (i % 32)) & 1).astype(bool)


def decode_u8(G: np.ndarray, N: int, missing_words: np.ndarray | None = None):
    """G: uint8 [M][ldg] dosage bytes. Returns (bytes int64 [M][N], missing bool [M][N]);
    bytes are 0 under a missing call."""
    G = np.asarray(G, dtype=np.uint8)
    vals = G[:, :N].astype(np.int64)
    missing = unpack_mask(missing_words, G.shape[0], N)
    vals = np.where(missing, 0, vals)
    return vals, missing


def marker_stats(units: np.ndarray, missing: np.ndarray):
    """Exact per-marker integers over observed calls, in decode units (counts or bytes).

    Returns n_obs, S = sum of units, S2 = sum of squared units (Python ints in int64
    arrays) and mean_units = S / n_obs as one correctly rounded float64 division
    (NaN when no call is observed).
    """
    obs = ~missing
    n_obs = obs.sum(axis=1).astype(np.int64)
    u = np.where(obs, units, 0).astype(np.int64)
    S = u.sum(axis=1)
    S2 = (u * u).sum(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean_units = np.where(n_obs > 0, S.astype(np.float64) / np.maximum(n_obs, 1), np.nan)
    return n_obs, S, S2, mean_units


def impute(units: np.ndarray, missing: np.ndarray, mean_units: np.ndarray, scale: float = 1.0):
    """Genotype values in allele-1 units (scale * units), a missing call replaced by the
    marker's observed mean. float64 [M][N]."""
    g = units.astype(np.float64)
    g = np.where(missing, mean_units[:, None], g)
    return scale * g
