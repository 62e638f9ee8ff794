"""SFT-domain demodulation on the GPU (fstat_sft_demod, fstat_sft_normalize)
against the oracles of the demodulation method and of the front end's
normalisation."""
import math

import numpy as np
import pytest

import synth
from oracle import demod as DM
from oracle import frontend as FE
from oracle import inject as I

pytestmark = pytest.mark.gpu

FS, N, F_H, N_SFT = 32.0, 4096, 10.0, 169        # 128 s SFTs of 32 Hz data, 6 h
T = N / FS


def _data():
    """Normalised SFTs (noise of sigma_r^2 = 1 per raw sample plus one
    injected signal), SFT times, the plan of the output grid, the injection."""
    raw = synth.PlanDesc(dt=1.0 / FS, n_data=N_SFT * N, f_het=F_H)
    plan = synth.PlanDesc(dt=0.5, n_data=int(N_SFT * T / 0.5), n_fft=1 << 16, f_het=F_H, max_templates=3)
    q_off = 1234
    inj = synth.random_injection(synth.SEED_BASE + 95, df=q_off / (plan.n_fft * plan.dt), fdot=-3e-10)
    inj.h0 = 0.1                                   # 2F about 400 at the signal
    s_raw = I.signal(inj, raw)
    h = 2.0 * np.real(s_raw * np.exp(2j * math.pi * F_H * np.arange(raw.n_data) / FS))
    k_h = int(round(F_H * T))
    sd = synth.SftDesc(sft_len=N, dt_raw=1.0 / FS, k_lo=k_h - 300, n_bins=601, k_het=k_h, band_bins=2,
                       dirichlet_terms=16, median_window=51)
    X = synth.sfts_of(h, np.arange(N_SFT), N, sd.k_lo, sd.n_bins, dtype=np.complex128)
    X = (X + synth.sft_noise(N_SFT, sd.n_bins, N, 1.0, synth.SEED_BASE + 96)) / math.sqrt(N)
    return X.astype(np.complex64), np.arange(N_SFT) * T, plan, sd, inj, q_off


def test_normalisation_matches_the_oracle():
    import torch
    import paper_0912_4255_gb300 as fs
    X, _, _, sd, _, _ = _data()
    got = fs.fstat_sft_normalize(sd, torch.from_numpy(X).cuda()).cpu().numpy()
    want = FE.normalize(X.astype(np.complex128), sd.median_window)
    assert np.abs(got - want).max() < 2e-5 * np.abs(want).max()


def test_demodulation_matches_the_oracle():
    """Three templates (the injection's and two others), 2F on the whole
    output grid on the GPU; the oracle on 48 random bins and a run of 40
    bins across the signal.  R15 metric <= 1e-4.  The bins at the ends of
    the grid reach outside the stored SFT bins: NaN and ERANGE."""
    import torch
    import paper_0912_4255_gb300 as fs
    X, t_sft, plan, sd, inj, q_off = _data()
    a, d = synth.random_sky(2, synth.SEED_BASE + 97)
    tm = synth.make_templates([inj.alpha, a[0], a[1]], [inj.delta, d[0], d[1]], [inj.fdot, 0.0, -1e-9], 0, 1)
    p = fs.Plan(plan, device=torch.device("cuda:0"))
    n_q = plan.n_fft
    out = fs.fstat_sft_demod(p, sd, torch.from_numpy(X).cuda(), torch.from_numpy(t_sft).cuda(),
                             fs.pack_templates(tm, device="cuda"), 0, n_q).cpu().numpy()
    df = 1.0 / (plan.n_fft * plan.dt)
    # the stored bins reach kappa_lo = k_lo + dk .. k_lo + n_bins - 1 - dk, Doppler of at most ~1.1e-4
    f_lo = (sd.k_lo + sd.dirichlet_terms) / T * (1 + 2e-4)
    f_hi = (sd.k_lo + sd.n_bins - 1 - sd.dirichlet_terms) / T * (1 - 2e-4)
    f = F_H + (np.arange(n_q) - n_q // 2) * df
    inside = (f > f_lo) & (f < f_hi)
    assert np.all(np.isfinite(out[:, inside]))
    assert fs.fstat_status(p, raise_error=False) == (0 if inside.all() else -2)
    g = synth.rng(5)
    qs = np.concatenate([g.choice(np.nonzero(inside)[0], 48, replace=False),
                         n_q // 2 + q_off + np.arange(-20, 20)])
    for i in range(3):
        want = DM.two_f(X.astype(np.complex128), sd, plan, t_sft, tm["alpha"][i], tm["delta"][i],
                        F_H + (qs - n_q // 2) * df, fdot=tm["fdot"][i])
        err = np.max(np.abs(out[i, qs] - want) / np.maximum(want, 4.0))
        assert err < 1e-4, (i, err)
    # the injection stands out at its own template and frequency
    assert int(np.argmax(out[0, inside])) == int(np.nonzero(inside)[0].searchsorted(n_q // 2 + q_off))


def test_demodulation_argument_errors():
    import torch
    import paper_0912_4255_gb300 as fs
    plan = synth.PlanDesc(dt=0.5, n_data=1000, n_fft=1 << 12, f_het=F_H, max_templates=1)
    p = fs.Plan(plan, device=torch.device("cuda:0"))
    sd = synth.SftDesc(sft_len=N, dt_raw=1.0 / FS, k_lo=1000, n_bins=20, k_het=1280, dirichlet_terms=16)
    X = torch.zeros((2, 20), dtype=torch.complex64, device="cuda")
    t = torch.zeros(2, dtype=torch.float64, device="cuda")
    tm = fs.pack_templates(synth.make_templates([1.0], [0.2], [0.0], 0, 1), device="cuda")
    with pytest.raises(fs.FstatError):                  # 2 dk + 1 > n_bins
        fs.fstat_sft_demod(p, sd, X, t, tm, 0, 16)


def test_no_bins_or_templates_is_a_no_op():
    import torch
    import paper_0912_4255_gb300 as fs
    X, t_sft, plan, sd, inj, q_off = _data()
    p = fs.Plan(plan, device=torch.device("cuda:0"))
    tm = fs.pack_templates(synth.make_templates([1.0], [0.2], [0.0], 0, 1), device="cuda")
    out = fs.fstat_sft_demod(p, sd, torch.from_numpy(X).cuda(), torch.from_numpy(t_sft).cuda(), tm, 100, 0)
    assert out.numel() == 0 and fs.fstat_status(p, raise_error=False) == 0
