"""Pins of the SFT front-end oracle (Sec. III.B) against closed forms, exact
transforms and brute force."""
import math

import numpy as np
import pytest

import synth
from oracle import frontend as FE

N, DT = 2048, 1.0 / 256.0            # 8 s SFTs at 256 Hz
T_SFT = N * DT
K_H, N1, DK, PAD = 400, 64, 16, 8    # f_h = 50 Hz, output interval 0.125 s


def _desc(**kw):
    d = synth.SftDesc(sft_len=N, dt_raw=DT, k_lo=K_H - N1 // 2 - DK - PAD, n_bins=N1 + 2 * (DK + PAD),
                      k_het=K_H, band_bins=N1, dirichlet_terms=DK, tukey_frac=0.1)
    return d.replace(**kw)


def test_dirichlet_kernel_special_values():
    """Eq. e9's P_{b,k}: 1 when the long bin is the SFT bin (y = 0), 0 at the
    other SFT bins (y a non-zero multiple of 2 pi), and at half a bin
    (b / M - k = 1/2 - j) the value -2i / (pi (1 - 2j))."""
    M = 6
    assert FE.dirichlet(5 * M, 5, M) == 1.0
    for j in (-3, -1, 1, 2):
        assert abs(FE.dirichlet(5 * M, 5 + j, M)) < 1e-15
    for j in (0, 1, -2):
        assert abs(FE.dirichlet(5 * M + M // 2, 5 + j, M) - (-2j / (math.pi * (1 - 2 * j)))) < 1e-15


def test_chunks_split_at_gaps_and_jitter():
    t = np.array([0, 1, 2, 5, 6, 7.5, 8.5]) * T_SFT
    assert FE.chunks(t, T_SFT) == [(0, 3), (3, 2), (5, 2)]
    t = np.array([0, 1 + 5e-7, 2 + 5e-7, 3 + 3e-6]) * T_SFT       # within / beyond 1e-6 T_SFT
    assert FE.chunks(t, T_SFT) == [(0, 3), (3, 1)]


def test_zero_sfts_normalise_to_zero():
    X = synth.sft_noise(3, 200, N, 1.0, 12).astype(np.complex128)
    X[1] = 0.0
    Xh = FE.normalize(X, 21)
    assert np.all(Xh[1] == 0) and np.all(np.isfinite(Xh))


def test_running_median_matches_brute_force_and_normalises():
    """Eq. dimlessSFTs1: interior bins take the plain median of their window;
    SFTs of different noise levels all come out with E|X^|^2 = 1 (median of
    an exponential variable = ln 2 x its mean; window 101: a few % scatter)."""
    X = synth.sft_noise(6, 2400, N, 1.0, 7).astype(np.complex128)
    X *= np.array([1.0, 3.0, 0.3, 10.0, 1.0, 2.0])[:, None]       # non-stationary
    S = FE.running_median_psd(X, 11)
    P = np.abs(X) ** 2
    for k in (5, 100, 2394):
        assert np.allclose(S[:, k], np.median(P[:, k - 5:k + 6], axis=1) / math.log(2))
    Xh = FE.normalize(X, 101)
    m = np.mean(np.abs(Xh) ** 2, axis=1)
    assert np.all(np.abs(m - 1.0) < 0.07), m          # sigma of each mean ~0.02, plus the window's noise


def test_on_grid_sinusoids_reproduce_the_heterodyned_series_exactly():
    """A sinusoid with a whole number of cycles per SFT occupies one bin of
    every SFT, so Eq. e9 is exact (only y = 0 terms).  Two such sinusoids in
    12 SFT slots with slots 4-5 missing (two chunks), the output starting 3
    samples before the first SFT: the series must be
    sum (A/2) e^{i (2 pi f t + phi)} e^{-2 pi i f_h (t - t_s)} x N / sqrt(N1)
    on both chunks (one phase reference: the chunk factor of
    Eq. hetStartCorr) and zero in the gap."""
    d = _desc()
    slots = np.array([0, 1, 2, 3, 6, 7, 8, 9, 10, 11])
    f = [(K_H + 5) / T_SFT, (K_H - 9) / T_SFT]
    A, ph = [2.0, 0.7], [0.3, -1.1]
    x_raw = synth.raw_sinusoids(12 * N, DT, f, A, ph)
    X = synth.sfts_of(x_raw, slots, N, d.k_lo, d.n_bins, dtype=np.complex128)
    dt_out = T_SFT / N1
    t_s = -3 * dt_out
    n_out = 3 + 12 * N1
    x = FE.sft_to_series(X, slots * T_SFT, d, t_s, n_out)
    t = t_s + np.arange(n_out) * dt_out
    want = sum(a / 2 * np.exp(1j * (2 * math.pi * fi * t + p)) for fi, a, p in zip(f, A, ph))
    want = want * np.exp(-2j * math.pi * (K_H / T_SFT) * (t - t_s)) * N / math.sqrt(N1)
    inside = np.zeros(n_out, bool)
    for a in slots:
        inside[3 + a * N1:3 + (a + 1) * N1] = True
    scale = np.abs(want).max()
    assert np.abs(x[inside] - want[inside]).max() < 1e-9 * scale
    assert np.all(x[~inside] == 0)


def _exact_chunk_series(x_raw, M, d):
    """Step 4 done exactly (the long DFT of the chunk's raw samples), then
    the same band selection, window and inverse transform as step 5."""
    Xl = np.fft.fft(x_raw[:M * N])
    n_out = d.band_bins * M
    m = np.arange(-n_out // 2, n_out // 2)
    spec = Xl[(d.k_het * M + m) % (M * N)] * FE.tukey(n_out, d.tukey_frac)
    return np.fft.ifft(np.fft.ifftshift(spec)) * n_out / math.sqrt(M * n_out)


@pytest.mark.parametrize("fo", [3.37, 3.5, -11.81])
def test_truncated_dirichlet_merge_near_the_signal(fo):
    """Sec. III.B.2: Eq. e9 keeps 2 dk + 1 kernel terms.  Near an off-bin
    sinusoid (long bins within one SFT bin of it) the dropped terms j > dk
    are SFT leakage |X| <= (A N / 2) / (pi j) times kernel values
    |P| <= 1 / (pi j); summed over both tails and the M SFTs they are at most
    (A N M / 2) 2 / (pi^2 dk), i.e. 1 / (pi dk) of the long transform's
    peak, which is at least 2/pi of A N M / 2.  (Over all N SFT bins and
    with the exact kernel (1 - e^{-iy}) / (N (1 - e^{-iy/N})) the merge is
    the long DFT itself; Eq. e75's large-N form differs from that kernel
    by about y / 2N, below 3 % at the outermost of these terms.)"""
    M = 6
    errs = []
    for dk in (4, 16, 40):
        d = _desc(dirichlet_terms=dk, k_lo=K_H - N1 // 2 - dk - PAD, n_bins=N1 + 2 * (dk + PAD))
        x_raw = synth.raw_sinusoids(M * N, DT, [(K_H + fo) / T_SFT], [1.0], [0.2])
        X = synth.sfts_of(x_raw, np.arange(M), N, d.k_lo, d.n_bins, dtype=np.complex128)
        b0 = int(round((K_H + fo) * M))
        b = np.arange(b0 - M, b0 + M + 1)
        Xb = FE.merge(X, d.k_lo, b, dk)
        Xl = np.fft.fft(x_raw)[b]
        err = np.abs(Xb - Xl).max() / np.abs(Xl).max()
        assert err < 1.0 / (math.pi * dk), (dk, err)
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


def test_merge_error_in_time_falls_with_the_kernel_length():
    """The series of step 5 from the truncated merge approaches the series
    from the exact long transform as dk grows (RMS over the chunk); the
    remaining error sits at the SFT boundaries, where each SFT's periodic
    extension is discontinuous."""
    M = 6
    rms, far = [], []
    for dk in (4, 16, 40):
        d = _desc(dirichlet_terms=dk, k_lo=K_H - N1 // 2 - dk - PAD, n_bins=N1 + 2 * (dk + PAD))
        x_raw = synth.raw_sinusoids(M * N, DT, [(K_H + 3.37) / T_SFT, (K_H - 11.81) / T_SFT],
                                    [1.0, 0.5], [0.2, 2.0])
        X = synth.sfts_of(x_raw, np.arange(M), N, d.k_lo, d.n_bins, dtype=np.complex128)
        z = FE.chunk_series(X, d.k_lo, K_H, N1, dk, d.tukey_frac)
        ze = _exact_chunk_series(x_raw, M, d)
        e = np.abs(z - ze)
        n = np.arange(len(z))
        dist = np.minimum(n % N1, N1 - n % N1)
        rms.append(math.sqrt(np.mean(e ** 2) / np.mean(np.abs(ze) ** 2)))
        far.append(e[dist > 4].max() / e.max())
    assert rms[0] > rms[1] > rms[2]
    assert max(far) < 0.5


def test_normalised_noise_has_the_window_mean_square():
    """Steps 2-5 on white noise: E|x_h|^2 = mean of the squared Tukey window
    (the scale 1 / sqrt(M N_out) with E|X^|^2 = 1)."""
    M = 8
    d = _desc(median_window=33, tukey_frac=0.2)
    X = synth.sft_noise(M, d.n_bins, N, 3.0, 11).astype(np.complex128)
    x = FE.sft_to_series(X, np.arange(M) * T_SFT, d, 0.0, M * N1)
    want = np.mean(FE.tukey(M * N1, 0.2) ** 2)
    assert abs(np.mean(np.abs(x) ** 2) / want - 1) < 0.1


def test_tukey_window_closed_forms():
    """Sec. III.B.5's band window, pinned by what defines a Tukey window
    rather than by re-evaluating its formula.  Sampled at x = (i + 1/2)/n
    with taper width e = frac/2 of the band on each side:
    * it is 1 on the flat part e <= x <= 1 - e and symmetric, w[i] = w[n-1-i];
    * it is 1/2 at the middle of each taper (x = e/2, which is a sample here);
    * on the rise it is the half-angle form sin^2(pi x / (2 e)), so samples
      at x and e - x add up to 1;
    * its mean is 1 - frac/2 exactly when n e is a whole number (the cosine
      part sums to zero over the midpoint samples of a half period);
    * frac = 1 is the Hann window sin^2(pi x); frac = 0 is all ones.
    A grid x = i/n, e = frac instead of frac/2, a flipped cosine sign or a
    missing mirrored fall each break at least one of these."""
    n, frac = 20, 0.3                       # e = 0.15 = 3 samples, x = e/2 at i = 1
    w = FE.tukey(n, frac)
    x = (np.arange(n) + 0.5) / n
    e = frac / 2
    assert np.allclose(w, w[::-1], atol=1e-15, rtol=0)
    assert np.all(w[(x >= e) & (x <= 1 - e)] == 1.0)
    assert abs(w[1] - 0.5) < 1e-15 and abs(w[n - 2] - 0.5) < 1e-15
    rise = x < e
    assert np.allclose(w[rise], np.sin(math.pi * x[rise] / (2 * e)) ** 2, atol=1e-15, rtol=0)
    assert abs(w[0] + w[2] - 1.0) < 1e-15
    assert np.all(np.diff(w[:4]) > 0) and 0 < w[0] < 0.5
    assert abs(w.mean() - (1 - frac / 2)) < 1e-15
    for n2, f2 in ((64, 0.25), (1000, 0.1), (36, 1.0 / 3.0)):
        assert abs(FE.tukey(n2, f2).mean() - (1 - f2 / 2)) < 1e-13
    xh = (np.arange(64) + 0.5) / 64
    assert np.allclose(FE.tukey(64, 1.0), np.sin(math.pi * xh) ** 2, atol=1e-15, rtol=0)
    assert np.all(FE.tukey(64, 0.0) == 1.0)


@pytest.mark.parametrize("taper", [5, 16])
def test_edge_taper_of_a_constant_chunk(taper):
    """Sec. III.B.6 (chunk stitching, optional taper at the chunk ends): a
    sinusoid at exactly the heterodyne frequency makes every chunk of x_h a
    constant (one SFT bin, Eq. e9 exact, Tukey window 1 at the band centre).
    With the taper, the first and last e samples of each chunk are that
    constant times the raised cosine sin^2(pi (i + 1/2) / (2 e)), i = 0..e-1
    at the start and mirrored at the end; the rest of the chunk and the gap
    are untouched.  The taper of e samples sums to e/2, and its samples i
    and e-1-i add up to 1.  A taper that starts at i instead of i + 1/2, a
    flipped cosine, or a missing or unmirrored end taper fails."""
    d = _desc()
    slots = np.array([0, 1, 2, 5, 6, 7])                 # two chunks of 3 SFTs
    x_raw = synth.raw_sinusoids(8 * N, DT, [K_H / T_SFT], [1.5], [0.4])
    X = synth.sfts_of(x_raw, slots, N, d.k_lo, d.n_bins, dtype=np.complex128)
    n_out = 8 * N1
    flat = FE.sft_to_series(X, slots * T_SFT, d, 0.0, n_out)
    tap = FE.sft_to_series(X, slots * T_SFT, d.replace(edge_taper=taper), 0.0, n_out)
    i = np.arange(taper)
    r = np.sin(math.pi * (i + 0.5) / (2 * taper)) ** 2
    assert abs(r.sum() - taper / 2) < 1e-12 and np.allclose(r + r[::-1], 1.0, atol=1e-15)
    for a, m in ((0, 3), (5, 3)):
        lo, hi = a * N1, (a + m) * N1
        c = flat[lo:hi]
        assert np.abs(c - c[0]).max() < 1e-9 * abs(c[0])      # the chunk is one constant
        ratio = tap[lo:hi] / c
        assert np.abs(ratio[:taper] - r).max() < 1e-12
        assert np.abs(ratio[-taper:] - r[::-1]).max() < 1e-12
        assert np.abs(ratio[taper:-taper] - 1.0).max() < 1e-12
    assert np.all(tap[3 * N1:5 * N1] == 0) and np.all(flat[3 * N1:5 * N1] == 0)
