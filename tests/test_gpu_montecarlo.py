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
