"""Monte Carlo of the statistic (the paper's validation of Sec. IV.B: 2F is
chi^2 with 4 degrees of freedom in Gaussian noise, non-central with the
optimal SNR^2 as non-centrality when a signal is present).

Realizations are consecutive 12 h spans of one long series, one template per
span (each template reads only its own samples), nearest-neighbour
resampling so that the resampled noise stays white."""
import math

import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import inject as I

pytestmark = pytest.mark.gpu

SPAN = 86400                         # 12 h at dt = 0.5 s


def _run(x, desc, n_real, alpha, delta):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc, device=dev)
    tm = synth.make_templates([alpha] * n_real, delta, 0.0, np.arange(n_real) * SPAN, SPAN)
    out = fs.fstat_compute(plan, torch.from_numpy(x).to(dev), fs.pack_templates(tm, device=dev))
    assert fs.fstat_status(plan, raise_error=False) == 0
    return out, tm


def test_noise_only_two_f_is_chi2_4():
    """256 realizations x 2^17 bins: mean 4, variance 8 and the tail
    probabilities P(2F > x) = e^{-x/2} (1 + x/2) of chi^2_4."""
    import torch
    n_real = 256
    desc = synth.tiny_plan(n_data=n_real * SPAN, max_templates=n_real)
    x = synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + 30)
    out, _ = _run(x, desc, n_real, 1.1, 0.4)
    v = out.double()
    mean, var = float(v.mean()), float(v.var())
    assert abs(mean - 4.0) < 0.01 and abs(var - 8.0) < 0.08, (mean, var)
    n = v.numel()
    for thr in (10.0, 20.0, 30.0):
        p = math.exp(-thr / 2) * (1 + thr / 2)
        got = float((v > thr).sum()) / n
        assert abs(got - p) < 6 * math.sqrt(p / (n / 3)) + 0.02 * p, (thr, got, p)


def test_injections_are_noncentral_chi2_4():
    """32 realizations of one continuous signal (rho = 20 over each span):
    at the injection bin E[2F] = lambda + 4 and Var = 8 + 4 lambda with
    lambda the oracle's noise-free 2F of that realization's template."""
    n_real = 32
    desc = synth.tiny_plan(n_data=n_real * SPAN, max_templates=n_real)
    df = 3000 / (desc.n_fft * desc.dt)
    inj = synth.random_injection(synth.SEED_BASE + 31, df=df)
    valid = I.valid_all(desc)
    # the amplitude of a rho = 20 signal over one 12 h span
    h0 = I.h0_for_rho(inj, desc.replace(n_data=SPAN), I.valid_all(desc.replace(n_data=SPAN)), 20.0)
    inj.h0 = h0
    s, _ = I.inject(np.zeros(desc.n_data), [inj], desc, valid)
    noise = synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + 32)
    x = (s + noise).astype(np.complex64)
    out, tm = _run(x, desc, n_real, inj.alpha, inj.delta)
    got = out.cpu().numpy().reshape(n_real, -1)
    q = desc.n_fft // 2 + 3000
    lam = np.array([F.resample_two_f(s.astype(np.complex128), tm[r], np.zeros((0, 2), np.int64), desc)[q]
                    for r in range(n_real)])
    z = (got[:, q] - lam - 4.0) / np.sqrt(8.0 + 4.0 * lam)
    assert lam.min() > 200
    assert abs(z.mean()) < 3.0 / math.sqrt(n_real), z.mean()
    assert 0.4 < z.var() < 1.8, z.var()


def test_stats_against_numpy():
    """fstat_stats on chi^2_4 values with NaN, +-inf and negative values
    mixed in and a length that leaves a ragged tail: counts and histogram
    exact, sums within FP32-partial rounding, and a second call adding
    to the first."""
    import torch
    import paper_0912_4255_gb300 as fs
    g = synth.rng(75)
    n = 3_000_003
    a = g.chisquare(4, size=n).astype(np.float32)
    a[::1001] = np.nan
    a[5::7919] = np.inf
    a[7::8191] = -np.inf
    a[11::12289] = -1.5
    a[-1] = 39.99999
    t = torch.from_numpy(a).cuda()
    acc = torch.zeros(6, dtype=torch.float64, device="cuda")
    hist = torch.zeros(40, dtype=torch.float64, device="cuda")
    thr = (10.0, 20.0, 30.0)
    for _ in range(2):
        fs.fstat_stats(t, acc, thr, hist, 1.0)
    torch.cuda.synchronize()
    fin = a[np.isfinite(a)].astype(np.float64)
    got = acc.cpu().numpy() / 2
    assert got[0] == fin.size
    assert abs(got[1] - fin.sum()) <= 1e-6 * abs(fin.sum())
    assert abs(got[2] - (fin * fin).sum()) <= 1e-6 * (fin * fin).sum()
    for i, th in enumerate(thr):
        assert got[3 + i] == np.count_nonzero(fin > th)
    x = fin[fin >= 0].astype(np.float32)
    b = np.floor(x / np.float32(1.0)).astype(np.int64)
    want = np.bincount(b[b < 40], minlength=40)
    assert np.array_equal(hist.cpu().numpy() / 2, want)
    # bins of width 2.5 (the quotient in FP32, as documented)
    hist5 = torch.zeros(16, dtype=torch.float64, device="cuda")
    acc1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    fs.fstat_stats(t, acc1, (), hist5, 2.5)
    b5 = np.floor(x / np.float32(2.5)).astype(np.int64)
    assert np.array_equal(hist5.cpu().numpy(), np.bincount(b5[b5 < 16], minlength=16))
    assert acc1.cpu().numpy()[0] == fin.size
