"""Per-band top-k candidates on the GPU against the oracle's selection:
bit-exact values and bins on spectra the oracle provides, and through the
whole path on an injected signal."""
import numpy as np
import pytest

import synth
from oracle import candidates as CA
from oracle import resample as R

from _gpu import injected_series, oracle_two_f, run_compute

pytestmark = pytest.mark.gpu


def _gpu_topk(a, band_len, k):
    import torch
    import paper_0912_4255_gb300 as fs
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    v, b = fs.fstat_topk(t, band_len, k, n_rows=a.shape[0])
    torch.cuda.synchronize()
    return v.cpu().numpy(), b.cpu().numpy()


@pytest.mark.parametrize("band_len,k", [(2048, 1), (4096, 7), (16384, 64), (65536, 16)])
def test_topk_matches_oracle_selection(band_len, k):
    """chi^2_4-like rows with planted peaks, heavy ties (values rounded to a
    coarse grid), a NaN row (an invalid template) and NaN bins."""
    g = synth.rng(71)
    a = g.chisquare(4, size=(5, 65536)).astype(np.float32)
    a[1] = np.round(a[1] * 2) / 2                 # many equal values
    a[2, 100:140] = 300.0 + np.arange(40)         # a cluster larger than k in one place
    a[3] = np.nan
    a[4, ::7] = np.nan
    v, b = _gpu_topk(a, band_len, k)
    ov, ob = CA.band_top_k(a.astype(np.float64), band_len, k)
    assert np.array_equal(v.astype(np.float64), ov)   # float32 values survive float64 exactly
    assert np.array_equal(b.astype(np.int64), ob)


@pytest.mark.parametrize("band_len,k", [(6144, 33), (10240, 64)])
def test_topk_bands_with_a_partial_sweep_step(band_len, k):
    """Bands of 3 and 5 sweeps of 2048 values (not whole steps of four):
    the last step of a band is partial.  Rows of 61440 values: noise, a
    slowly rising ramp (many values pass the bound, the buffer fills over
    several steps) and a row that is NaN but for a few bins."""
    g = synth.rng(72)
    a = g.chisquare(4, size=(3, 61440)).astype(np.float32)
    a[1] = (np.arange(61440) % band_len).astype(np.float32) * 0.01 + g.random(61440).astype(np.float32)
    a[2] = np.nan
    a[2, ::5000] = 7.0
    v, b = _gpu_topk(a, band_len, k)
    ov, ob = CA.band_top_k(a.astype(np.float64), band_len, k)
    assert np.array_equal(v.astype(np.float64), ov)
    assert np.array_equal(b.astype(np.int64), ob)


def test_topk_rising_band_merges_repeatedly():
    """A strictly increasing band: every value passes the running bound, so
    the candidate buffer fills and merges on every step."""
    a = np.arange(2 * 65536, dtype=np.float32).reshape(2, 65536)
    a[1] = a[1][::-1]
    v, b = _gpu_topk(a, 65536, 64)
    ov, ob = CA.band_top_k(a.astype(np.float64), 65536, 64)
    assert np.array_equal(v.astype(np.float64), ov) and np.array_equal(b.astype(np.int64), ob)


def test_topk_after_compute_finds_the_injection():
    """The whole path: 2F of a 2^17 FFT with an injected signal, then the
    candidates; against the oracle's candidates of the oracle's own 2F (the
    loudest bin of the band with the signal, and the candidate values to
    the parity tolerance at the bins the GPU chose)."""
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=100_000, n_fft=1 << 17, interp=R.SINC, f_het=80.0,
                       max_templates=1)
    inj = synth.random_injection(72, df=0.2)
    x, _ = injected_series(d, 73, [inj])
    tm = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, d.n_data)
    got, rc = run_compute(d, x, tm)
    assert rc == 0
    ref = oracle_two_f(d, x, tm[0])
    v, b = _gpu_topk(got, 16384, 8)
    ov, ob = CA.band_top_k(ref[None, :], 16384, 8)
    loud = int(np.argmax(ov[0, :, 0]))
    assert b[0, loud, 0] == ob[0, loud, 0] and ov[0, loud, 0] > 100
    chosen = ref[b[0].reshape(-1)]
    assert np.max(np.abs(v[0].reshape(-1) - chosen) / np.maximum(chosen, 4.0)) <= 1e-4


def test_topk_into_given_tensors_on_a_second_stream():
    """The output tensors of one call reused by the next, on a stream other
    than the default one (as a search pipelines its chunks): the same values
    and bins as separate calls, and wrong output tensors are refused."""
    import torch
    import paper_0912_4255_gb300 as fs
    g = synth.rng(74)
    a = torch.from_numpy(g.chisquare(4, size=(3, 16384)).astype(np.float32)).cuda()
    want_v, want_b = fs.fstat_topk(a, 4096, 8, n_rows=3)
    s = torch.cuda.Stream()
    v = torch.empty((3, 4, 8), dtype=torch.float32, device="cuda")
    b = torch.empty((3, 4, 8), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        for _ in range(2):
            rv, rb = fs.fstat_topk(a, 4096, 8, n_rows=3, stream=s, val=v, bins=b)
    s.synchronize()
    assert rv is v and rb is b
    assert torch.equal(v, want_v) and torch.equal(b, want_b)
    with pytest.raises(ValueError):
        fs.fstat_topk(a, 4096, 8, n_rows=3, val=v[:2], bins=b)
    with pytest.raises(ValueError):
        fs.fstat_topk(a, 4096, 8, n_rows=3, val=v, bins=b.float())
