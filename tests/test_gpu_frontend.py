"""SFT front end on the GPU (fstat_sft_series) against the oracle of
Sec. III.B, element by element, and against the closed form of bin-centred
sinusoids at realistic sizes."""
import math

import numpy as np
import pytest

import synth
from oracle import frontend as FE

pytestmark = pytest.mark.gpu


def _gpu(d, X, t_sft, t_start, n_out):
    import torch
    import paper_0912_4255_gb300 as fs
    x = fs.fstat_sft_series(d, torch.from_numpy(np.ascontiguousarray(X)).cuda(), t_sft, t_start, n_out)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128)


def _case(N, n1, dk, pad, slots, n_slots, seed, **kw):
    k_h = N // 5
    d = synth.SftDesc(sft_len=N, dt_raw=1.0 / 256.0, k_lo=k_h - n1 // 2 - dk - pad,
                      n_bins=n1 + 2 * (dk + pad), k_het=k_h, band_bins=n1, dirichlet_terms=dk, **kw)
    t_len = d.t_sft
    g = synth.rng(seed)
    f = k_h / t_len + g.uniform(-0.4, 0.4, 3) * n1 / t_len
    x_raw = synth.raw_sinusoids(n_slots * N, d.dt_raw, f, [3.0, 1.0, 0.5], g.uniform(0, 6, 3))
    x_raw = x_raw + g.normal(0.0, 1.0, x_raw.size)
    X = synth.sfts_of(x_raw, slots, N, d.k_lo, d.n_bins)
    return d, X, np.asarray(slots, float) * t_len


@pytest.mark.parametrize("kw", [
    dict(n1=64, dk=16, pad=8, median_window=33, tukey_frac=0.1, edge_taper=5),
    dict(n1=90, dk=5, pad=20, median_window=0, tukey_frac=0.0, edge_taper=0),
    dict(n1=16, dk=0, pad=3, median_window=7, tukey_frac=1.0, edge_taper=1000),
])
def test_series_matches_the_oracle(kw):
    """Ragged chunks of 1, 3, 7 and 2 SFTs with gaps between them; the output
    starts 3 samples before the first SFT and runs 5 samples past the last."""
    N = 2048
    slots = [0, 2, 3, 4, 7, 8, 9, 10, 11, 12, 13, 16, 17]
    n1, dk, pad = kw.pop("n1"), kw.pop("dk"), kw.pop("pad")
    d, X, t = _case(N, n1, dk, pad, slots, 18, 70 + n1, **kw)
    dt_out = d.t_sft / n1
    t_s = -3 * dt_out
    n_out = 3 + 18 * n1 + 5
    want = FE.sft_to_series(X.astype(np.complex128), t, d, t_s, n_out)
    got = _gpu(d, X, t, t_s, n_out)
    scale = np.abs(want).max()
    err = np.abs(got - want).max() / scale
    assert err < 3e-5, err
    assert np.array_equal(got == 0, want == 0)          # gaps and the margins


def test_zero_sft_and_jittered_times():
    """An SFT of zeros normalises to zeros (no NaN), and start times
    jittered by less than 1e-6 T_SFT still form one chunk, as in the
    oracle."""
    N = 2048
    slots = [0, 1, 2, 3, 4, 5]
    d, X, t = _case(N, 64, 16, 8, slots, 6, 77, median_window=33, tukey_frac=0.1)
    X[2] = 0
    t = t + np.array([0, 3e-7, -2e-7, 4e-7, 0, 1e-7]) * d.t_sft
    n_out = 6 * 64
    want = FE.sft_to_series(X.astype(np.complex128), t, d, 0.0, n_out)
    got = _gpu(d, X, t, 0.0, n_out)
    assert np.all(np.isfinite(got))
    assert np.abs(got - want).max() < 3e-5 * np.abs(want).max()


def test_bin_centred_sinusoids_at_full_band_size():
    """N1 = 3600 band bins per SFT (2 Hz at T_SFT = 1800 s: dt_out = 0.5 s),
    chunks of 24 and 9 SFTs: sinusoids with whole cycles per SFT come out
    as (A/2) e^{i (2 pi f t + phi)} e^{-2 pi i f_h (t - t_s)} N / sqrt(N1) to
    FP32 accuracy (Eq. e9 is exact for them)."""
    N, dt = 1 << 15, 1.0 / 16.0                          # 2048 s SFTs at 16 Hz
    n1, dk, pad = 3600, 16, 8
    k_h = 9000
    d = synth.SftDesc(sft_len=N, dt_raw=dt, k_lo=k_h - n1 // 2 - dk - pad, n_bins=n1 + 2 * (dk + pad),
                      k_het=k_h, band_bins=n1, dirichlet_terms=dk, tukey_frac=0.05)
    slots = np.array(list(range(24)) + list(range(26, 35)))
    t_len = d.t_sft
    f = [(k_h + 700) / t_len, (k_h - 1311) / t_len]
    A, ph = [2.0, 0.5], [0.4, -2.0]
    x_raw = synth.raw_sinusoids(35 * N, dt, f, A, ph)
    X = synth.sfts_of(x_raw, slots, N, d.k_lo, d.n_bins)
    n_out = 35 * n1
    got = _gpu(d, X, slots * t_len, 0.0, n_out)
    tt = np.arange(n_out) * (t_len / n1)
    want = sum(a / 2 * np.exp(1j * (2 * math.pi * fi * tt + p)) for fi, a, p in zip(f, A, ph))
    want = want * np.exp(-2j * math.pi * (k_h / t_len) * tt) * N / math.sqrt(n1)
    inside = np.zeros(n_out, bool)
    for a in slots:
        inside[a * n1:(a + 1) * n1] = True
    scale = np.abs(want).max()
    assert np.abs(got[inside] - want[inside]).max() < 2e-4 * scale
    assert np.all(got[~inside] == 0)


def test_no_sfts_gives_zeros():
    import torch
    import paper_0912_4255_gb300 as fs
    d, X, t = _case(2048, 64, 16, 8, [0], 1, 5)
    x = torch.full((300,), 7.0, dtype=torch.complex64, device="cuda")
    fs.fstat_sft_series(d, torch.from_numpy(X[:0].copy()).cuda(), t[:0], 0.0, 300, x_h=x)
    torch.cuda.synchronize()
    assert bool((x == 0).all())
