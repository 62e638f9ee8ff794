"""Pins of the SFT-domain demodulation oracle (the method of Sec. IV.A's
comparison) against brute force, the chi^2_4 statistics and the resampling
method on the same signal."""
import math

import numpy as np

import synth
from oracle import demod as DM
from oracle import fstat as F
from oracle import inject as I


def test_bin_centred_signal_without_doppler_equals_the_direct_sum():
    """No Roemer delay (AU = R = 0), no spindown, a sinusoid with whole
    cycles per SFT evaluated at its own frequency: the linear phase within
    each SFT is exact and only the y = 0 kernel term is non-zero, so F_a and
    F_b (hence 2F) equal the brute-force sums over the raw samples with a, b
    held at each SFT's midpoint."""
    N, dt = 512, 1.0 / 64.0
    T = N * dt
    eph = synth.Ephem(au_m=0.0)
    det = synth.Detector(radius_m=0.0)
    plan = synth.PlanDesc(dt=dt, n_data=40 * N, det=det, eph=eph)
    k0 = 100
    sd = synth.SftDesc(sft_len=N, dt_raw=dt, k_lo=k0 - 20, n_bins=41, k_het=k0, band_bins=2,
                       dirichlet_terms=16)
    slots = np.array([0, 1, 2, 5, 6, 9, 10, 11, 30, 39])
    x = synth.raw_sinusoids(40 * N, dt, [k0 / T], [1.0], [0.7])
    X = synth.sfts_of(x, slots, N, sd.k_lo, sd.n_bins, dtype=np.complex128)
    got = DM.two_f(X, sd, plan, slots * T, 1.1, 0.3, k0 / T)[0]
    # brute force
    tau, rate, a, b = DM.sft_midpoint_terms(plan, sd, slots * T, 1.1, 0.3)
    assert np.all(rate == 0)
    Fa = Fb = 0.0j
    for i, s in enumerate(slots):
        t = (s * N + np.arange(N)) * dt
        z = np.sum(x[s * N:(s + 1) * N] * np.exp(-2j * math.pi * (k0 / T) * (t - plan.t_start)))
        Fa += a[i] * z
        Fb += b[i] * z
    A, B, C = np.sum(a * a), np.sum(b * b), np.sum(a * b)
    want = 2 * (B * abs(Fa) ** 2 + A * abs(Fb) ** 2 - 2 * C * (Fa * np.conj(Fb)).real) / (A * B - C * C)
    assert abs(got - want) < 1e-9 * want


def test_normalised_noise_is_chi2_4():
    """Normalised noise SFTs (E|X^|^2 = 1): 2F at 400 frequencies one SFT
    bin apart has the chi^2_4 mean 4 and variance 8 (3 sigma bounds)."""
    N, dt = 4096, 1.0 / 32.0
    T = N * dt
    plan = synth.PlanDesc(dt=dt, n_data=60 * N)
    sd = synth.SftDesc(sft_len=N, dt_raw=dt, k_lo=1000, n_bins=460, k_het=1230, band_bins=2,
                       dirichlet_terms=16)
    X = synth.sft_noise(60, sd.n_bins, N, 1.0, 90).astype(np.complex128) / math.sqrt(N)
    f = (1030 + np.arange(400) + 0.37) / T
    v = DM.two_f(X, sd, plan, np.arange(60) * T, 2.0, -0.5, f, fdot=-1e-10)
    assert abs(v.mean() - 4) < 3 * math.sqrt(8 / 400), v.mean()
    assert abs(v.var() - 8) < 3 * math.sqrt(384 / 400), v.var()


def test_demodulation_agrees_with_resampling_on_one_signal():
    """The two methods of Sec. IV.A on the same injected signal: its raw
    real strain at 32 Hz cut into 128 s SFTs (normalised by the raw noise
    level sigma_r^2 = 1: X^ = X / sqrt(N)) for the demodulation, and the
    heterodyned 2 Hz series of the same strain (noise variance
    sigma_r^2 B / f_s per sample) for the resampling; both at the true
    template and the signal's frequency recover rho^2 to a few %."""
    fs, N = 32.0, 4096
    T = N / fs
    f_h = 10.0
    n_sft = 169                                   # 6 h
    raw = synth.PlanDesc(dt=1.0 / fs, n_data=n_sft * N, f_het=f_h)
    out = synth.PlanDesc(dt=0.5, n_data=int(n_sft * T / 0.5), n_fft=1 << 16, f_het=f_h, interp=synth.SINC,
                         taps=8, sigma2=2.0 / fs)
    q_off = 1234
    inj = synth.random_injection(synth.SEED_BASE + 91, df=q_off / (out.n_fft * out.dt), fdot=-3e-10)
    inj.h0 = I.h0_for_rho(inj, out, I.valid_all(out), 20.0)
    rho2 = I.rho2(inj, out, I.valid_all(out))
    # resampling on the heterodyned series
    s_out = I.signal(inj, out)
    tm = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, out.n_data)[0]
    r_res = F.resample_two_f(s_out, tm, np.zeros((0, 2), np.int64), out)[out.n_fft // 2 + q_off]
    # demodulation on SFTs of the raw strain 2 Re[s e^{2 pi i f_h (t - t_s)}]
    s_raw = I.signal(inj, raw)
    t = np.arange(raw.n_data) / fs
    h = 2.0 * np.real(s_raw * np.exp(2j * math.pi * f_h * t))
    k_h = int(round(f_h * T))
    sd = synth.SftDesc(sft_len=N, dt_raw=1.0 / fs, k_lo=k_h - 300, n_bins=601, k_het=k_h, band_bins=2,
                       dirichlet_terms=16)
    X = synth.sfts_of(h, np.arange(n_sft), N, sd.k_lo, sd.n_bins, dtype=np.complex128) / math.sqrt(N)
    r_dem = DM.two_f(X, sd, raw, np.arange(n_sft) * T, inj.alpha, inj.delta, f_h + inj.df, fdot=inj.fdot)[0]
    assert abs(r_res / rho2 - 1) < 0.03, r_res / rho2
    assert abs(r_dem / rho2 - 1) < 0.05, r_dem / rho2
