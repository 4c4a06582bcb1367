"""GPU parity of the decode step and of panel preparation against the FP64 oracle.

Decode must match bit for bit (integer statistics, the FP64 mean, the operand values);
the panel (Q, Y_res, s) must match to FP64 rounding.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_21095_gb300 as tg
import synth

pytestmark = pytest.mark.gpu


def bf16_rn(x):
    """Nearest bf16 value (ties to even) of float64 values, computed exactly in float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _decode(tgctx, G, N, enc, prec, missing=None):
    M = G.shape[0]
    lda = synth.round_up(N, 64)
    dev = G.device
    if prec == tg.TG_PREC_SPLIT_BF16:
        A = torch.full((M, lda), 7.0, dtype=torch.bfloat16, device=dev)
        shift = torch.full((M,), 7.0, dtype=torch.float32, device=dev)
    else:
        A = torch.full((M, lda), 7.0, dtype=torch.float32, device=dev)
        shift = None
    n_obs = torch.zeros(M, dtype=torch.int32, device=dev)
    S = torch.zeros(M, dtype=torch.int64, device=dev)
    S2 = torch.zeros(M, dtype=torch.int64, device=dev)
    mean = torch.zeros(M, dtype=torch.float64, device=dev)
    tg.tg_decode_block(tgctx, G, N, M, enc, prec, A, shift, missing=missing, n_obs=n_obs, S=S,
                       S2=S2, mean=mean)
    torch.cuda.synchronize()
    a = A.double().cpu().numpy()
    c = None if shift is None else shift.double().cpu().numpy()
    return a, c, n_obs.cpu().numpy(), S.cpu().numpy(), S2.cpu().numpy(), mean.cpu().numpy()


def _check_operand(a, shift, units, miss, mean, prec, N, enc):
    """FP32: codes, float(mean) at missing calls. Split: the row centred on its shift c (the
    mean rounded to multiples of 1/128 for 2-bit calls, to integers for dosage bytes, ties to
    even, 0 without observed calls), exact at observed calls, bf16(mean - c) at missing ones."""
    assert np.all(a[:, N:] == 0)
    obs = ~miss
    m_imp = np.where(np.isnan(mean), 0.0, mean)
    if prec == tg.TG_PREC_SPLIT_BF16:
        grid = 128.0 if enc == tg.TG_ENC_2BIT else 1.0
        c = np.where(np.isnan(mean), 0.0, np.rint(m_imp * grid) / grid)
        assert np.array_equal(shift, c)
        assert np.all(np.abs(m_imp - c) <= 0.5 / grid)
        exp_obs = np.where(obs, units - c[:, None], 0)
        assert np.array_equal(np.where(obs, a[:, :N], 0), exp_obs)
        h = bf16_rn(m_imp - c)
        assert np.array_equal(np.where(miss, a[:, :N], 0), np.where(miss, h[:, None], 0))
    else:
        assert shift is None
        assert np.array_equal(np.where(obs, a[:, :N], 0), np.where(obs, units, 0).astype(np.float64))
        f = m_imp.astype(np.float32).astype(np.float64)
        assert np.array_equal(np.where(miss, a[:, :N], 0), np.where(miss, f[:, None], 0))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 63, 64, 65, 130, 1999, 23001, 24576, 24577, 49153])
@pytest.mark.parametrize("prec", [tg.TG_PREC_SPLIT_BF16, tg.TG_PREC_FP32])
def test_decode_2bit_bit_exact(tgctx, N, prec):
    g = torch.Generator().manual_seed(N)
    M = 37
    counts = torch.randint(0, 3, (M, N), generator=g, dtype=torch.int8)
    miss = torch.rand(M, N, generator=g) < 0.1
    miss[0] = True                      # no observed call
    counts[1] = 2
    miss[1] = False                     # monomorphic
    G = synth.pack_2bit(counts, miss).cuda()
    a, c, n, S, S2, mean = _decode(tgctx, G, N, tg.TG_ENC_2BIT, prec)
    units, m = oracle.decode_2bit(G.cpu().numpy(), N)
    n0, S0, S20, mean0 = oracle.marker_stats(units, m)
    assert np.array_equal(n, n0) and np.array_equal(S, S0) and np.array_equal(S2, S20)
    assert np.array_equal(np.isnan(mean), np.isnan(mean0))
    assert np.array_equal(mean[~np.isnan(mean)], mean0[~np.isnan(mean0)])   # bit-exact FP64
    _check_operand(a, c, units, m, mean, prec, N, tg.TG_ENC_2BIT)


def test_decode_2bit_every_byte_value(tgctx):
    N = 4 * 256
    row = np.arange(256, dtype=np.uint8)
    G = np.zeros((3, synth.round_up(256, 16)), dtype=np.uint8)
    G[0, :256] = row
    G[1, :256] = row[::-1]
    G[2, :256] = np.roll(row, 77)
    Gt = torch.from_numpy(G).cuda()
    a, c, n, S, S2, mean = _decode(tgctx, Gt, N, tg.TG_ENC_2BIT, tg.TG_PREC_SPLIT_BF16)
    units, m = oracle.decode_2bit(G, N)
    n0, S0, S20, mean0 = oracle.marker_stats(units, m)
    assert np.array_equal(n, n0) and np.array_equal(S, S0) and np.array_equal(S2, S20)
    assert np.array_equal(mean, mean0)
    _check_operand(a, c, units, m, mean, tg.TG_PREC_SPLIT_BF16, N, tg.TG_ENC_2BIT)


# split-form rows of N <= 24,576 and <= 49,152 take the block-per-row kernels, larger N the
# warp-per-row kernel
@pytest.mark.parametrize("N", [1, 15, 16, 17, 33, 2000, 23000, 24576, 24577, 49152, 49153])
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("prec", [tg.TG_PREC_SPLIT_BF16, tg.TG_PREC_FP32])
def test_decode_u8_bit_exact(tgctx, N, masked, prec):
    g = torch.Generator().manual_seed(1000 + N)
    M = 21
    freq = synth.maf(5, N, M)
    G = synth.dosage_bytes(5, N, freq, N).cuda()
    missing = synth.missing_words(5, N, M, N, 0.2).cuda() if masked else None
    if masked:
        missing[0] = -1                 # every call missing
    a, c, n, S, S2, mean = _decode(tgctx, G, N, tg.TG_ENC_U8_DOSAGE, prec, missing)
    units, m = oracle.decode_u8(G.cpu().numpy(), N, None if missing is None else missing.cpu().numpy())
    n0, S0, S20, mean0 = oracle.marker_stats(units, m)
    assert np.array_equal(n, n0) and np.array_equal(S, S0) and np.array_equal(S2, S20)
    ok = ~np.isnan(mean0)
    assert np.array_equal(np.isnan(mean), ~ok) and np.array_equal(mean[ok], mean0[ok])
    _check_operand(a, c, units, m, mean, prec, N, tg.TG_ENC_U8_DOSAGE)
    del g


# ---------------------------------------------------------------- panel

def _panel_inputs(N, P, n_cov, seed, extra=None):
    cov = synth.covariates(seed, N, n_cov)
    if extra is not None:
        cov = torch.cat([cov, extra(cov)], 0)
    Yt = synth.phenotypes(seed, cov, P)
    return cov, Yt


@pytest.mark.parametrize("N,P,n_cov", [(2000, 37, 4), (1999, 5, 0), (23000, 3, 19), (300, 600, 9)])
def test_panel_matches_oracle(tgctx, N, P, n_cov):
    cov, Yt = _panel_inputs(N, P, n_cov, seed=N + P)
    Yt[0] = 2.5                                              # constant phenotype
    if n_cov:
        Yt[1] = cov[0].float()                               # inside the covariate span
        cov[0] = Yt[1].double()
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda() if n_cov else None)
    try:
        N_, P_, q, df = tg.tg_panel_info(panel)
        ref = oracle.prepare_panel(Yt.numpy().T.astype(np.float64), cov.numpy().T if n_cov else None)
        assert (N_, P_, q, df) == (N, P, ref["q"], ref["df"])
        Q = tg.tg_panel_Q(panel).cpu().numpy().T[:, :q]
        Qo = ref["Q"]
        assert np.allclose(Q, Qo, atol=1e-12, rtol=0)
        Yres, s = tg.tg_panel_Yres(panel)
        Yres = Yres.cpu().numpy().T
        s = s.cpu().numpy()
        scale = np.linalg.norm(ref["Y"] - ref["Y"].mean(0), axis=0).max()
        assert np.allclose(Yres, ref["Yres"], atol=1e-11 * scale, rtol=0)
        ok = ref["pheno_ok"]
        assert np.allclose(s[ok], ref["s"][ok], rtol=1e-12)
        assert not ok[0] and (not ok[1] if n_cov else True)
    finally:
        tg.tg_panel_free(panel)


def test_panel_rank_detection(tgctx):
    N, P = 500, 4
    cov = synth.covariates(3, N, 4)
    cov = torch.cat([cov, cov[1:2], torch.full((1, N), 3.0, dtype=torch.float64),
                     (2 * cov[0] - cov[3]).unsqueeze(0)], 0)
    Yt = synth.phenotypes(3, cov[:4], P)
    panel = tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    try:
        _, _, q, df = tg.tg_panel_info(panel)
        assert q == 5 and df == N - 6
    finally:
        tg.tg_panel_free(panel)


def test_panel_rejects_nonfinite_and_rank(tgctx):
    N, P = 100, 3
    cov = synth.covariates(4, N, 2)
    Yt = synth.phenotypes(4, cov, P)
    Yt[1, 17] = float("nan")
    with pytest.raises(tg.TgError) as e:
        tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    assert e.value.status == tg.TG_ERR_NONFINITE
    Yt = synth.phenotypes(4, cov, P)
    cov[1, 3] = float("inf")
    with pytest.raises(tg.TgError) as e:
        tg.tg_prepare_panel(tgctx, Yt.cuda(), N, P, cov.cuda())
    assert e.value.status == tg.TG_ERR_NONFINITE
    small = synth.covariates(5, 3, 2)
    with pytest.raises(tg.TgError) as e:
        tg.tg_prepare_panel(tgctx, synth.phenotypes(5, small, 2).cuda(), 3, 2, small.cuda())
    assert e.value.status == tg.TG_ERR_RANK
