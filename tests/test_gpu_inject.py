"""fstat_inject against the oracle's signal model (Eqs. 1-4 with the
detector-tensor antenna functions), and through the whole path."""

import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import inject as I

pytestmark = pytest.mark.gpu

SPAN = 86400


def _injections():
    """Three signals with different sky positions, frequencies, spindowns
    and orientations; the second and third overlap."""
    out = []
    for k, (df, fdot, fddot) in enumerate([(0.0458, 0.0, 0.0), (-0.31, -2e-9, 0.0), (0.47, 3e-10, 4e-15)]):
        out.append(synth.random_injection(synth.SEED_BASE + 40 + k, df=df, fdot=fdot, fddot=fddot))
    return out


def _oracle(desc, injs, h0, starts, lens):
    s = np.zeros(desc.n_data, np.complex128)
    n = np.arange(desc.n_data)
    for inj, h, a, l in zip(injs, h0, starts, lens):
        s += np.where((n >= a) & (n < a + l), I.signal(inj, desc, h0=h), 0.0)
    return s


def _plan(desc):
    import torch
    import paper_0912_4255_gb300 as fs
    return fs.Plan(desc, device=torch.device("cuda:0"))


def test_signals_match_the_oracle():
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.tiny_plan(n_data=2 * SPAN + 777)
    injs = _injections()
    h0 = [1.0, 0.7, 1.3]
    starts, lens = [1000, 80001, 120003], [SPAN - 1234, SPAN - 1, 52000]
    rec = synth.injection_records(injs, h0, starts, lens)
    plan = _plan(desc)
    noise = synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + 44)
    x = torch.from_numpy(noise).cuda()
    fs.fstat_inject(plan, x, rec)
    assert fs.fstat_status(plan, raise_error=False) == 0
    got = x.cpu().numpy().astype(np.complex128) - noise.astype(np.complex128)
    want = _oracle(desc, injs, h0, starts, lens)
    amp = np.abs(want).max()
    err = np.abs(got - want).max() / amp
    # FP32 evaluation: phase offsets held to ~6e-8 cycles, amplitudes and the
    # stored sum noise + signal to FP32 rounding (~6e-7 of the amplitude)
    assert err < 3e-6, err
    # samples outside every span are untouched, bit for bit
    n = np.arange(desc.n_data)
    inside = np.zeros(desc.n_data, bool)
    for a, l in zip(starts, lens):
        inside |= (n >= a) & (n < a + l)
    assert np.array_equal(x.cpu().numpy()[~inside], noise[~inside])


def test_invalid_records_set_the_status_and_are_skipped():
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.tiny_plan(n_data=SPAN)
    injs = _injections()[:2]
    rec = synth.injection_records(injs, 1.0, [0, 100], [1000, 1000])
    rec["delta"][1] = 2.0                      # |delta| > pi/2
    plan = _plan(desc)
    x = torch.zeros(desc.n_data, dtype=torch.complex64, device="cuda:0")
    fs.fstat_inject(plan, x, rec)
    assert fs.fstat_status(plan, raise_error=False) == -1           # EINVAL
    want = _oracle(desc, injs[:1], [1.0], [0], [1000])
    got = x.cpu().numpy()
    assert np.abs(got - want).max() < 3e-6 * np.abs(want).max()
    # a span past the end of the data: ERANGE, nothing written
    rec = synth.injection_records(injs[:1], 1.0, [SPAN - 10], [20])
    x.zero_()
    fs.fstat_inject(plan, x, rec)
    assert fs.fstat_status(plan, raise_error=False) == -2
    assert not bool(x.abs().max() > 0)


def test_injected_signal_through_the_path():
    """2F of a GPU-injected signal equals the oracle's 2F of the oracle's
    injection of the same signal (R15 metric, every bin)."""
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.tiny_plan()
    inj = synth.random_injection(synth.SEED_BASE + 45, df=3000 / (desc.n_fft * desc.dt))
    h0 = I.h0_for_rho(inj, desc, I.valid_all(desc), 20.0)
    plan = _plan(desc)
    x = torch.zeros(desc.n_data, dtype=torch.complex64, device="cuda:0")
    fs.fstat_inject(plan, x, synth.injection_records([inj], h0, 0, desc.n_data))
    tm = synth.make_templates(inj.alpha, inj.delta, 0.0, 0, desc.n_data)
    out = fs.fstat_compute(plan, x, fs.pack_templates(tm, device=x.device)).cpu().numpy()
    assert fs.fstat_status(plan, raise_error=False) == 0
    s = I.signal(inj, desc, h0=h0)
    want = F.resample_two_f(s, tm[0], np.zeros((0, 2), np.int64), desc)
    err = np.max(np.abs(out - want) / np.maximum(want, 4.0))
    assert err < 1e-4, err
    q = desc.n_fft // 2 + 3000
    assert want[q] > 300 and int(np.argmax(out)) == q


def test_no_injections_is_a_no_op():
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.tiny_plan(n_data=1000)
    plan = _plan(desc)
    x = torch.ones(desc.n_data, dtype=torch.complex64, device="cuda:0")
    fs.fstat_inject(plan, x, synth.injection_records([], 1.0, 0, 0))
    fs.fstat_inject(plan, x, synth.injection_records(_injections()[:1], 1.0, 0, 0))   # empty span
    assert fs.fstat_status(plan, raise_error=False) == 0
    assert bool((x == 1).all())
