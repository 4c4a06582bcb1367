"""Named synthetic workloads with the shapes and value distributions of the paper's benchmark.

The paper's cohort (about 23,000 samples, 8.9 million markers; Section 3.1) is not
available, so these seeded sets stand in for it: hard calls ~ Binomial(2, maf) with
maf ~ U(0.01, 0.5), MCAR missing calls, N(0,1) covariates plus an intercept, and
Gaussian phenotypes with covariate effects and planted causal markers at h2 = 0.02 each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import gwas


@dataclass(frozen=True)
class Workload:
    name: str
    N: int              # samples
    M: int              # markers in the whole scan
    P: int              # phenotypes
    n_cov: int          # covariate columns besides the intercept
    encoding: str       # "2bit" (PLINK-style hard calls) or "u8" (8-bit dosages)
    missing: float      # MCAR missing-call rate
    seed: int
    block: int          # markers per streamed block
    causal_per_pheno: int = 0   # causal markers drawn per phenotype (small panels)
    planted: int = 0            # planted (marker, phenotype) pairs (large panels)
    h2: float = 0.02

    @property
    def n_blocks(self) -> int:
        return (self.M + self.block - 1) // self.block

    def block_range(self, b: int):
        m0 = b * self.block
        return m0, min(self.M, m0 + self.block)


WORKLOADS = {
    w.name: w
    for w in (
        Workload("n2000_m10000_p16_c5_2bit", N=2000, M=10_000, P=16, n_cov=4, encoding="2bit",
                 missing=0.01, seed=1, block=10_000, causal_per_pheno=5),
        Workload("n23000_m1000000_p2048_c10_2bit", N=23_000, M=1_000_000, P=2048, n_cov=9,
                 encoding="2bit", missing=0.005, seed=2, block=65_536, planted=50),
        Workload("n23000_m8900000_p20480_c20_u8", N=23_000, M=8_900_000, P=20_480, n_cov=19,
                 encoding="u8", missing=0.0, seed=5, block=65_536, planted=50),
        Workload("n23000_m500000_12panels_p8192_2bit", N=23_000, M=500_000, P=8192, n_cov=9,
                 encoding="2bit", missing=0.005, seed=4, block=65_536, planted=50),
    )
}

# The batched workload: 12 phenotype panels of uneven size over the same samples and covariates.
BATCHED_PANELS = (17, 256, 1000, 3500, 1, 64, 128, 300, 500, 626, 800, 1000)
assert sum(BATCHED_PANELS) == 8192


def ragged_blocks(seed: int, M: int, lo: int = 1000, hi: int = 65_536):
    """Block sizes ~ U[lo, hi] drawn until they cover M markers; a short remainder is merged into
    the last block while that stays <= hi (else it is its own block)."""
    g = gwas.generator("cpu", seed, 99, 0)
    sizes, total = [], 0
    while total < M:
        b = int(torch.randint(lo, hi + 1, (1,), generator=g))
        b = min(b, M - total)
        if b < lo and sizes and sizes[-1] + b <= hi:
            sizes[-1] += b
        else:
            sizes.append(b)
        total += b
    return sizes


def make_block(w: Workload, b: int, device="cpu", with_truth: bool = False) -> dict:
    """Genotype block b of workload w: packed rows G (uint8 [Mb][ldg]) and, for dosages
    with a missing rate, the bit-packed mask (int32 [Mb][ceil(N/32)])."""
    m0, m1 = w.block_range(b)
    Mb = m1 - m0
    f = gwas.maf(w.seed, b, Mb, device=device)
    out = {"m0": m0, "M": Mb, "maf": f, "missing": None}
    if w.encoding == "2bit":
        counts, miss = gwas.hard_calls(w.seed, b, f, w.N, w.missing, device=device)
        out["G"] = gwas.pack_2bit(counts, miss)
        out["ldg"] = out["G"].shape[1]
        if with_truth:
            out["truth"] = counts.to(torch.float64)
    else:
        out["G"] = gwas.dosage_bytes(w.seed, b, f, w.N, device=device)
        out["ldg"] = out["G"].shape[1]
        if w.missing > 0:
            out["missing"] = gwas.missing_words(w.seed, b, Mb, w.N, w.missing, device=device)
        if with_truth:
            out["truth"] = out["G"][:, : w.N].to(torch.float64) * (2.0 / 255.0)
    return out


def make_ragged_block(w: Workload, index: int, M: int, device="cpu") -> torch.Tensor:
    """Packed genotypes of the index-th ragged block (M markers), drawn with its own keys."""
    f = gwas.maf(w.seed, 1000 + index, M, device=device)
    if w.encoding == "2bit":
        counts, miss = gwas.hard_calls(w.seed, 1000 + index, f, w.N, w.missing, device=device)
        return gwas.pack_2bit(counts, miss)
    return gwas.dosage_bytes(w.seed, 1000 + index, f, w.N, device=device)


def _planted_pairs(w: Workload, n_blocks: int):
    """(global marker, phenotype) pairs carrying a planted effect."""
    g = gwas.generator("cpu", w.seed, 77, 0)
    if w.causal_per_pheno:
        idx = gwas.causal_choice(w.seed, min(w.M, n_blocks * w.block), w.P, w.causal_per_pheno)
        return [(int(idx[p, k]), p) for p in range(w.P) for k in range(w.causal_per_pheno)]
    span = min(w.M, n_blocks * w.block)
    loci = torch.randperm(span, generator=g)[: w.planted]
    phen = torch.randint(0, w.P, (w.planted,), generator=g)
    return [(int(m), int(p)) for m, p in zip(loci, phen)]


def make_panel(w: Workload, device="cpu", planted_blocks: int = 1) -> dict:
    """Covariates (float64 [n_cov][N], column-major N x n_cov) and phenotypes
    (float32 [P][N], column-major N x P) with planted effects placed in the first
    `planted_blocks` genotype blocks."""
    cov_t = gwas.covariates(w.seed, w.N, w.n_cov, device=device)
    pairs = _planted_pairs(w, planted_blocks)
    by_block = {}
    for m, p in pairs:
        by_block.setdefault(m // w.block, []).append((m, p))
    planted = []
    for b, lst in sorted(by_block.items()):
        blk = make_block(w, b, device=device, with_truth=True)
        for m, p in lst:
            j = m - blk["m0"]
            fr = float(blk["maf"][j])
            beta = math.sqrt(w.h2 / (2.0 * fr * (1.0 - fr)))
            planted.append((p, blk["truth"][j], beta))
    Yt = gwas.phenotypes(w.seed, cov_t, w.P, planted, device=device)
    return {"cov_t": cov_t, "Yt": Yt, "pairs": pairs}
