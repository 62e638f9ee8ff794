"""Output band (fstat_set_band) and the band-doubling remedy of Sec. V.B."""
import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import inject as I

from _gpu import MODES

pytestmark = pytest.mark.gpu


def _setup(desc, n_t=3, seed=60):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = torch.device("cuda:0")
    x = torch.from_numpy(synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + seed)).to(dev)
    a, d = synth.random_sky(n_t, synth.SEED_BASE + seed + 1)
    tm = synth.make_templates(a, d, np.linspace(-1e-9, 0, n_t), 0, desc.n_data)
    return fs, dev, x, tm


@pytest.mark.parametrize("mode", ["split", "fused", "persistent", "split_n2_1024"])
def test_band_is_the_slice_of_the_full_output(mode):
    """Bit-exact: the band's values are the full output's values of the same
    bins, every template packed at index * band length.  split_n2_1024 runs
    the split path with N1 = 2^7, N2 = 2^10 (the row length of the search-sized
    FFT)."""
    desc = synth.tiny_plan(interp=synth.SINC, taps=8, max_templates=3)
    fs, dev, x, tm = _setup(desc)
    plan = fs.Plan(desc, device=dev)
    if mode == "split_n2_1024":
        plan.set_tuning(mode=MODES["split"], log2_n1=7)
    else:
        plan.set_tuning(mode=MODES[mode])
    td = fs.pack_templates(tm, device=dev)
    full = fs.fstat_compute(plan, x, td).cpu().numpy().reshape(3, -1)
    n = desc.n_fft
    for lo, hi in [(n // 4, 3 * n // 4), (5, n - 3), (12345, 12346), (0, n)]:
        plan.set_band(lo, hi)
        assert plan.band() == (lo, hi)
        out = fs.fstat_compute(plan, x, td)
        assert fs.fstat_status(plan, raise_error=False) == 0
        assert out.numel() == 3 * (hi - lo)
        np.testing.assert_array_equal(out.cpu().numpy().reshape(3, -1), full[:, lo:hi])


def test_band_arguments_and_invalid_templates():
    import paper_0912_4255_gb300 as fs
    desc = synth.tiny_plan(max_templates=2)
    fs_, dev, x, tm = _setup(desc, n_t=2)
    plan = fs.Plan(desc, device=dev)
    for lo, hi in [(-1, 10), (10, 10), (0, desc.n_fft + 1)]:
        with pytest.raises(fs.FstatError):
            plan.set_band(lo, hi)
    n = desc.n_fft
    plan.set_band(n // 4, 3 * n // 4)
    tm["span_len"][1] = desc.n_data + 1             # invalid span: NaN fill of its band only
    out = fs.fstat_compute(plan, x, fs.pack_templates(tm, device=dev)).cpu().numpy().reshape(2, -1)
    assert fs.fstat_status(plan, raise_error=False) == -2
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1]))
    # a template with its own n_fft under a partial band: ENOTSUP
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    tm = synth.make_templates([1.0], 0.3, 0.0, 0, desc.n_data, n_fft=n // 2)
    out = fs.fstat_compute(plan, x, fs.pack_templates(tm, device=dev), None,
                           torch_empty(n // 2, dev))
    assert fs.fstat_status(plan, raise_error=False) == -6


def torch_empty(n, dev):
    import torch
    return torch.full((n,), 0.0, dtype=torch.float32, device=dev)


def test_band_doubling_recovers_the_interpolation_loss():
    """Sec. V.B: near the top of the band the windowed-sinc resampling loses
    power (here 8-tap Lanczos at df = 0.9 Hz, dt = 0.5 s: 10 % in the
    oracle); the same signal in data sampled twice as fast, searched over
    the doubled band with only its central half kept, comes out at full
    power (1.000 in the oracle).  Both searches are compared with the
    oracle's 2F of the same data."""
    import torch
    import paper_0912_4255_gb300 as fs
    dev = torch.device("cuda:0")
    q_off = 58982                                   # df = q_off / 65536 s = 0.89999 Hz
    res = {}
    for dt, n_fft in [(0.5, 1 << 17), (0.25, 1 << 18)]:
        desc = synth.tiny_plan(dt=dt, n_data=int(43200 / dt), n_fft=n_fft, interp=synth.SINC, taps=8)
        inj = synth.random_injection(synth.SEED_BASE + 62, df=q_off / (n_fft * dt))
        valid = I.valid_all(desc)
        h0 = I.h0_for_rho(inj, desc, valid, 20.0)
        s = I.signal(inj, desc, h0=h0)
        tm = synth.make_templates(inj.alpha, inj.delta, 0.0, 0, desc.n_data)
        plan = fs.Plan(desc, device=dev)
        lo = n_fft // 4 if dt == 0.25 else 0
        if dt == 0.25:
            plan.keep_lower_half()
        out = fs.fstat_compute(plan, torch.from_numpy(s.astype(np.complex64)).to(dev),
                               fs.pack_templates(tm, device=dev)).cpu().numpy()
        assert fs.fstat_status(plan, raise_error=False) == 0
        want = F.resample_two_f(s, tm[0], np.zeros((0, 2), np.int64), desc)[lo:lo + out.size]
        assert np.max(np.abs(out - want) / np.maximum(want, 4.0)) < 1e-4
        q = n_fft // 2 + q_off - lo
        res[dt] = out[q] / 400.0
    assert res[0.5] < 0.92, res                     # the loss near the band top
    assert res[0.25] > 0.99, res                    # recovered in the kept half
