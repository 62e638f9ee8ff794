"""The single-precision device math written out by hand in the resampler,
on the GPU, against exact (FP64) values and against CUDA's sincospif:

* sincospi_small: sin and cos of pi x, |x| <= 1/4, Taylor series to x^9 and
  x^10 (truncation below 2e-9) evaluated by Horner's rule in FP32;
* expm2pi: exp(-2 pi i r), |r| <= 1/2, by exact quarter turns and
  sincospi_small of the remainder;
* the 8-tap windowed sinc of step 4 of Sec. III.A.2 (Lanczos window and
  plain truncation), whose weights use the approximate reciprocal
  rcp.approx.ftz.f32 (relative error below 2^-22 by the PTX definition),
  against the oracle's FP64 interpolation of the same samples.

Bounds (stated, and checked over a dense grid plus random points):
sincospi_small and expm2pi within 2.5e-7 absolute of the exact values and
within 2.5e-7 of CUDA's sincospif; the sine relative error below 2.5e-7;
the interpolant within 1e-6 of sum_i |w_i| |x_i| of the exact one."""
import numpy as np
import pytest

import synth
from oracle import resample as R

pytestmark = pytest.mark.gpu


def _run(which, x, aux=None):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
    ad = None if aux is None else torch.from_numpy(np.ascontiguousarray(aux, np.complex64)).to(dev)
    out = fs.fstat_selftest_math(which, xd, ad)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_sincospi_small_against_exact_and_cuda():
    g = synth.rng(1)
    x = np.concatenate([np.linspace(-0.25, 0.25, 1 << 20), g.uniform(-0.25, 0.25, 1 << 18),
                        [0.0, 1e-30, -1e-20, 1e-7, 0.25, -0.25]]).astype(np.float32)
    xs = x.astype(np.float64)
    got = _run("sincospi_small", x)
    cuda = _run("sincospif", x)
    s, c = np.sin(np.pi * xs), np.cos(np.pi * xs)
    assert np.abs(got[:, 0] - s).max() <= 2.5e-7
    assert np.abs(got[:, 1] - c).max() <= 2.5e-7
    nz = np.abs(xs) > 0
    assert (np.abs(got[nz, 0] - s[nz]) / np.abs(s[nz])).max() <= 2.5e-7
    assert np.abs(got - cuda).max() <= 2.5e-7
    assert got[np.nonzero(xs == 0)[0][0], 0] == 0.0 and got[np.nonzero(xs == 0)[0][0], 1] == 1.0


def test_expm2pi_against_exact():
    g = synth.rng(2)
    r = np.concatenate([np.linspace(-0.5, 0.5, 1 << 20), g.uniform(-0.5, 0.5, 1 << 18),
                        [0.0, 0.125, 0.25, -0.25, 0.375, 0.5, -0.5]]).astype(np.float32)
    got = _run("expm2pi", r)
    want = np.exp(-2j * np.pi * r.astype(np.float64))
    err = np.abs(got[:, 0] + 1j * got[:, 1] - want)
    assert err.max() <= 2.5e-7
    cuda = _run("sincospif", (2 * r.astype(np.float64)).astype(np.float32))
    assert np.abs(got[:, 0] - cuda[:, 1]).max() <= 2.5e-7 and np.abs(got[:, 1] + cuda[:, 0]).max() <= 2.5e-7


@pytest.mark.parametrize("window", [R.WIN_LANCZOS, R.WIN_RECT])
def test_sinc8_weights_against_exact_interpolation(window):
    g = synth.rng(3)
    n = 4096
    aux = (g.normal(size=n) + 1j * g.normal(size=n)).astype(np.complex64)
    base = np.arange(1, n - 2, dtype=np.float64)
    u = np.concatenate([
        g.uniform(0.0, n - 0.6, 1 << 17),                     # anywhere, edges included
        base, base + 0.5, base + 1e-7, base - 1e-6, base + 0.999,
        np.linspace(0.0, 8.0, 4097)]).astype(np.float32)
    u = u[u < n - 0.6]
    uu = u.astype(np.float64)
    got = _run("sinc8_lanczos" if window == R.WIN_LANCZOS else "sinc8_rect", u, aux)
    valid = np.ones(n, bool)
    want = R.interpolate(aux.astype(np.complex128), uu, valid, R.SINC, 8, window)
    # scale: sum of |w_i| |x_i| over the taps
    half, bas = 4, np.floor(uu).astype(np.int64)
    scale = np.zeros_like(uu)
    for i in range(8):
        j = bas - half + 1 + i
        d = uu - j
        w = np.sinc(d) * (np.sinc(d / half) if window == R.WIN_LANCZOS else 1.0)
        ok = (j >= 0) & (j < n)
        scale[ok] += np.abs(w[ok]) * np.abs(aux[j[ok]])
    err = np.abs(got[:, 0] + 1j * got[:, 1] - want) / scale
    assert err.max() <= 1e-6, float(err.max())
