"""Draws of genotypes, covariates and phenotypes with a fixed, regenerable seed scheme.

Every draw is keyed by (workload seed, stream id, block id, chunk id) through a
SplitMix64 mix (Steele, Lea & Flood 2014), so any genotype block can be
regenerated on its own, on any device, without drawing the blocks before it.
Draws on a CUDA device and on the CPU give different numbers (different torch
generators); a test always hands the same tensors to both sides of a comparison.
"""
from __future__ import annotations

import torch

_MASK64 = (1 << 64) - 1

# stream ids
_S_MAF, _S_CALLS, _S_MISS, _S_COV, _S_NOISE, _S_COVEFF, _S_CAUSAL, _S_JITTER, _S_MASK = range(1, 10)

# Markers are drawn in fixed chunks so that the numbers do not depend on how a
# caller batches the work.
_CHUNK = 4096

# PLINK 1 .bed (SNP-major) 2-bit field per allele-1 count; 0b01 marks a missing call.
_COUNT_TO_BED = (0b11, 0b10, 0b00)
BED_MISSING = 0b01


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


def block_seed(*keys: int) -> int:
    """SplitMix64 finaliser folded over the keys; returns a 63-bit seed."""
    z = 0x9E3779B97F4A7C15
    for k in keys:
        z = (z + (int(k) & _MASK64) * 0xBF58476D1CE4E5B9 + 0x9E3779B97F4A7C15) & _MASK64
        z ^= z >> 30
        z = (z * 0xBF58476D1CE4E5B9) & _MASK64
        z ^= z >> 27
        z = (z * 0x94D049BB133111EB) & _MASK64
        z ^= z >> 31
    return z & ((1 << 63) - 1)


def generator(device, *keys: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(block_seed(*keys))
    return g


def maf(seed: int, block: int, M: int, device="cpu", lo: float = 0.01, hi: float = 0.5) -> torch.Tensor:
    """Minor-allele frequencies ~ U(lo, hi), float64 [M]."""
    g = generator(device, seed, _S_MAF, block)
    return lo + (hi - lo) * torch.rand(M, generator=g, device=device, dtype=torch.float64)


def hard_calls(seed: int, block: int, freq: torch.Tensor, N: int, missing_rate: float = 0.0,
               device="cpu"):
    """Allele-1 counts ~ Binomial(2, freq) and an MCAR missing mask.

    Returns (counts int8 [M][N] in {0,1,2}, missing bool [M][N]). The counts under
    a missing call are kept (they are the truth a planted effect is built from).
    """
    M = freq.numel()
    counts = torch.empty(M, N, dtype=torch.int8, device=device)
    missing = torch.zeros(M, N, dtype=torch.bool, device=device)
    for c0 in range(0, M, _CHUNK):
        c1 = min(M, c0 + _CHUNK)
        g = generator(device, seed, _S_CALLS, block, c0 // _CHUNK)
        p = freq[c0:c1].to(device=device, dtype=torch.float32).unsqueeze(1)
        u = torch.rand(2, c1 - c0, N, generator=g, device=device)
        counts[c0:c1] = (u[0] < p).to(torch.int8) + (u[1] < p).to(torch.int8)
        if missing_rate > 0:
            gm = generator(device, seed, _S_MISS, block, c0 // _CHUNK)
            missing[c0:c1] = torch.rand(c1 - c0, N, generator=gm, device=device) < missing_rate
    return counts, missing


def pack_2bit(counts: torch.Tensor, missing: torch.Tensor | None = None, ldg: int | None = None) -> torch.Tensor:
    """PLINK 1 .bed SNP-major packing: sample i in bits 2(i%4)..2(i%4)+1 of byte i//4.

    Field values: count 2 -> 0b00, 1 -> 0b10, 0 -> 0b11, missing -> 0b01. Trailing
    fields of the last byte and bytes beyond ceil(N/4) (up to the row stride) are 0.
    """
    M, N = counts.shape
    nb = (N + 3) // 4
    ldg = ldg if ldg is not None else round_up(max(nb, 1), 16)
    assert ldg >= nb
    table = torch.tensor(_COUNT_TO_BED, dtype=torch.int32, device=counts.device)
    f = table[counts.long().clamp(0, 2)]
    if missing is not None:
        f = torch.where(missing, torch.full_like(f, BED_MISSING), f)
    pad = 4 * nb - N
    if pad:
        f = torch.cat([f, torch.zeros(M, pad, dtype=f.dtype, device=f.device)], dim=1)
    f = f.view(M, nb, 4)
    b = f[..., 0] | (f[..., 1] << 2) | (f[..., 2] << 4) | (f[..., 3] << 6)
    out = torch.zeros(M, ldg, dtype=torch.uint8, device=counts.device)
    out[:, :nb] = b.to(torch.uint8)
    return out


def dosage_bytes(seed: int, block: int, freq: torch.Tensor, N: int, jitter: float = 8.0,
                 ldg: int | None = None, device="cpu") -> torch.Tensor:
    """BGEN-like 8-bit dosages: b = clamp(round(127.5*g + U(-jitter, jitter)), 0, 255), g ~ Bin(2, freq).

    Byte b stands for the allele-1 dosage 2b/255. Returns uint8 [M][ldg], zero padded.
    """
    M = freq.numel()
    ldg = ldg if ldg is not None else round_up(max(N, 1), 16)
    out = torch.zeros(M, ldg, dtype=torch.uint8, device=device)
    for c0 in range(0, M, _CHUNK):
        c1 = min(M, c0 + _CHUNK)
        g = generator(device, seed, _S_CALLS, block, c0 // _CHUNK)
        p = freq[c0:c1].to(device=device, dtype=torch.float32).unsqueeze(1)
        u = torch.rand(2, c1 - c0, N, generator=g, device=device)
        cnt = (u[0] < p).to(torch.float32) + (u[1] < p).to(torch.float32)
        gj = generator(device, seed, _S_JITTER, block, c0 // _CHUNK)
        e = (torch.rand(c1 - c0, N, generator=gj, device=device) * 2.0 - 1.0) * jitter
        out[c0:c1, :N] = torch.clamp(torch.round(127.5 * cnt + e), 0, 255).to(torch.uint8)
    return out


def missing_words(seed: int, block: int, M: int, N: int, rate: float, device="cpu") -> torch.Tensor:
    """Bit-packed MCAR mask: bit (i % 32) of int32 word i // 32 of row j is set when call (j, i) is missing.

    Returns int32 [M][ceil(N/32)] (bits beyond N are 0).
    """
    W = (N + 31) // 32
    out = torch.zeros(M, W, dtype=torch.int32, device=device)
    for c0 in range(0, M, _CHUNK):
        c1 = min(M, c0 + _CHUNK)
        g = generator(device, seed, _S_MASK, block, c0 // _CHUNK)
        miss = torch.rand(c1 - c0, N, generator=g, device=device) < rate
        pad = W * 32 - N
        if pad:
            miss = torch.cat([miss, torch.zeros(c1 - c0, pad, dtype=torch.bool, device=device)], 1)
        bits = miss.view(c1 - c0, W, 32).to(torch.int64)
        shifts = torch.arange(32, device=device, dtype=torch.int64)
        words = (bits << shifts).sum(-1)
        out[c0:c1] = torch.where(words >= 2 ** 31, words - 2 ** 32, words).to(torch.int32)
    return out


def covariates(seed: int, N: int, n_cov: int, device="cpu") -> torch.Tensor:
    """n_cov N(0,1) covariate columns (the intercept is not included). float64, stored
    column-major: tensor [n_cov][N], so column k is row k (leading dimension N)."""
    g = generator(device, seed, _S_COV, 0)
    return torch.randn(n_cov, N, generator=g, device=device, dtype=torch.float64)


def phenotypes(seed: int, cov_t: torch.Tensor, P: int, planted=(), device="cpu",
               cov_effect_sd: float = 1.0) -> torch.Tensor:
    """Phenotype panel: y_p = gamma_p0 + C gamma_p + sum over planted (p, g, b) of b*g + eps.

    gamma ~ N(0, cov_effect_sd^2), eps ~ N(0, 1). `planted` is a sequence of
    (pheno index, genotype vector float64 [N], effect size). Returns float32 stored
    column-major: tensor [P][N], so phenotype p is row p (leading dimension N).
    """
    n_cov, N = cov_t.shape
    gc = generator(device, seed, _S_COVEFF, 0)
    gam = torch.randn(P, n_cov + 1, generator=gc, device=device, dtype=torch.float64) * cov_effect_sd
    y = torch.empty(P, N, dtype=torch.float32, device=device)
    ct = cov_t.to(device)
    for p0 in range(0, P, 1024):
        p1 = min(P, p0 + 1024)
        gn = generator(device, seed, _S_NOISE, p0 // 1024)
        blk = gam[p0:p1, :1] + gam[p0:p1, 1:] @ ct
        blk = blk + torch.randn(p1 - p0, N, generator=gn, device=device, dtype=torch.float64)
        y[p0:p1] = blk.to(torch.float32)
    for p, gvec, b in planted:
        y[p] = (y[p].double() + float(b) * gvec.to(device=device, dtype=torch.float64)).float()
    return y


def causal_choice(seed: int, M: int, P: int, per_pheno: int, device="cpu") -> torch.Tensor:
    """Causal marker indices: `per_pheno` distinct markers per phenotype, int64 [P][per_pheno]."""
    g = generator("cpu", seed, _S_CAUSAL, 0)
    idx = torch.stack([torch.randperm(M, generator=g)[:per_pheno] for _ in range(P)])
    return idx.to(device)
