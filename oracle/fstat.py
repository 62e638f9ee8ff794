"""The resampling F-statistic and direct demodulation (FP64, test oracle).

Procedure of Sec. III.A.2 (steps 1-7), in the paper's order:

 1. start from the heterodyned series x_h(t^k) on the regular detector grid;
 2. correct for the detector-frame heterodyne (Eq. absorb);
 3. compute T^k(t_b^k) (Eq. 21);
 4. interpolate z(T^k(t_b^k));
 5. a(t_b^k), b(t_b^k);
 6. FFT the two weighted series of Eqs. 19-20 -> F_a, F_b;
 7. the F-statistic, Eq. 6.

Readings of points the paper leaves open or garbles (each is pinned by a
``-m "not gpu"`` test):

* heterodyne sign: x_h = x exp(-2 pi i f_h (t - t_start)) (so that the
  995 Hz example of Sec. III.A.1 lands at DC) and the correction is
  z = x_h exp(-2 pi i f_h t_m); a signal at f_h + df then peaks at +df;
* spindown sign: the demodulation multiplies by exp(-i Phi_s), the conjugate
  of the signal's spindown phase (Eq. 7 with Eq. 5);
* Phi_s is the exact barycentric polynomial 2 pi sum_s f^(s) tau^(s+1)/(s+1)!
  with tau = t_b - t_start (Eq. 4 in barycentric time; Eq. 4pt1 is its
  first-order expansion in t_m), here to s = 2 (fdot, fddot);
* the heterodyne correction uses t_m at T^k, i.e. tau_k = t_b^k - T^k
  (Eq. phi-s-explain), applied after interpolating x_h (identical to the
  paper's order in the continuum);
* a and b are evaluated analytically at T^k instead of being interpolated;
* 2F for unit-free complex data: with A = sum m a^2, B = sum m b^2,
  C = sum m a b, D = A B - C^2 (Eqs. 9-10 as sums) and sigma^2 = E|n|^2 per
  complex sample, 2F = 2 (B|Fa|^2 + A|Fb|^2 - 2 C Re(Fa Fb*)) / (sigma^2 D),
  which is chi^2 with 4 degrees of freedom in Gaussian noise (Sec. IV.B);
* output order: ascending frequency offset, bin q <-> df = (q - N/2)/(N dt)
  (the FFT's DC/+f/-f order of Sec. V.A rotated by N/2).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, resample, timemap


def two_f(Fa, Fb, A, B, C, sigma2):
    """2F from F_a, F_b and the antenna-pattern sums (Eq. 6, complex-data
    normalisation)."""
    D = A * B - C * C
    return 2.0 * (B * np.abs(Fa) ** 2 + A * np.abs(Fb) ** 2
                  - 2.0 * C * np.real(Fa * np.conj(Fb))) / (sigma2 * D)


def _fddot(tmpl):
    """Second spindown of a template record (0 for records without it)."""
    names = getattr(getattr(tmpl, "dtype", None), "names", None) or ()
    return float(tmpl["fddot"]) if "fddot" in names else 0.0


def _frac(x):
    return x - np.floor(x)


def resampled_series(x_h, tmpl, gaps, plan):
    """Steps 1-5: the weighted series w_a, w_b on the barycentric grid and
    the sums A, B, C.  Returns a dict with every intermediate."""
    a_, d_ = float(tmpl["alpha"]), float(tmpl["delta"])
    fdot = float(tmpl["fdot"])
    fddot = _fddot(tmpl)
    tb, T, n_b = timemap.resample_times(tmpl, plan)
    u = resample.fractional_index(T, plan)
    valid = resample.valid_samples(plan.n_data, int(tmpl["span_start"]),
                                   int(tmpl["span_len"]), gaps)
    m = resample.mask(u, valid)
    z = resample.interpolate(x_h, u, valid, plan.interp, plan.taps, plan.window)
    # t_m(T^k) of Eq. phi-s-explain, evaluated at T^k: equal to t_b^k - T^k
    # by Eq. 21, but the difference of the two absolute times carries the
    # rounding of T (1 ulp = 4.7e-10 s at 30 d, 3e-6 rad at f_h = 1 kHz)
    tau = geometry.roemer_delay(T, a_, d_, plan.det, plan.eph)
    tau_b = tb - plan.t_start
    # phase in cycles, reduced mod 1 before the complex exponential
    cyc = _frac(plan.f_het * tau) + _frac(0.5 * fdot * tau_b * tau_b) + _frac(fddot * tau_b ** 3 / 6.0)
    y = m * z * np.exp(-2j * np.pi * cyc)
    a, b = geometry.beam_ab(T, a_, d_, plan.det, plan.eph)
    return dict(tb=tb, T=T, u=u, m=m, z=z, y=y, a=a, b=b, n_b=n_b,
                wa=a * y, wb=b * y,
                A=float(np.sum(m * a * a)), B=float(np.sum(m * b * b)),
                C=float(np.sum(m * a * b)))


def resample_two_f(x_h, tmpl, gaps, plan, n_fft=None, return_parts=False):
    """Steps 1-7: 2F in every bin of an n_fft-point FFT, ascending frequency
    offset from f_h (bin q <-> df = (q - n_fft/2)/(n_fft dt))."""
    n_fft = int(n_fft or plan.n_fft)
    r = resampled_series(x_h, tmpl, gaps, plan)
    if r["n_b"] > n_fft:
        raise ValueError("n_fft smaller than the resampled length")
    wa = np.zeros(n_fft, np.complex128)
    wb = np.zeros(n_fft, np.complex128)
    wa[:r["n_b"]] = r["wa"]
    wb[:r["n_b"]] = r["wb"]
    Fa = np.fft.fftshift(np.fft.fft(wa))
    Fb = np.fft.fftshift(np.fft.fft(wb))
    out = two_f(Fa, Fb, r["A"], r["B"], r["C"], plan.sigma2)
    if return_parts:
        r.update(Fa=Fa, Fb=Fb, two_f=out)
        return r
    return out


def bin_frequencies(n_fft, dt):
    """Frequency offset of each output bin (ascending)."""
    return (np.arange(n_fft) - n_fft // 2) / (n_fft * dt)


def direct_two_f(x_h, tmpl, gaps, plan, df):
    """Direct demodulation (Eqs. 7-8 as sums over the valid detector samples):
    F_a(df) = sum_n a(t_n) x_h[n] exp(-2 pi i [f_h t_m(t_n) + df tau_n
    + fdot tau_n^2 / 2 + fddot tau_n^3 / 6]), tau_n = t_n - t_start + t_m(t_n);
    F_b alike; 2F as in ``two_f``.  O(N) per frequency; no resampling."""
    a_, d_ = float(tmpl["alpha"]), float(tmpl["delta"])
    fdot = float(tmpl["fdot"])
    fddot = _fddot(tmpl)
    valid = resample.valid_samples(plan.n_data, int(tmpl["span_start"]),
                                   int(tmpl["span_len"]), gaps)
    n = np.nonzero(valid)[0]
    t = plan.t_start + n * plan.dt
    tm = geometry.roemer_delay(t, a_, d_, plan.det, plan.eph)
    tau = t - plan.t_start + tm
    a, b = geometry.beam_ab(t, a_, d_, plan.det, plan.eph)
    cyc = _frac(plan.f_het * tm) + _frac(0.5 * fdot * tau * tau) + _frac(fddot * tau ** 3 / 6.0)
    base = np.asarray(x_h, np.complex128)[n] * np.exp(-2j * np.pi * cyc)
    df = np.atleast_1d(np.asarray(df, dtype=np.float64))
    Fa = np.empty(df.size, np.complex128)
    Fb = np.empty(df.size, np.complex128)
    for i, f in enumerate(df):
        e = np.exp(-2j * np.pi * _frac(f * tau))
        Fa[i] = np.sum(a * base * e)
        Fb[i] = np.sum(b * base * e)
    A, B, C = float(np.sum(a * a)), float(np.sum(b * b)), float(np.sum(a * b))
    return two_f(Fa, Fb, A, B, C, plan.sigma2)


def single_bin_two_f(x_h, tmpl, gaps, plan, df):
    """2F of the resampled series at one continuous frequency offset df:
    F_a(df) = sum_k w_a[k] exp(-2 pi i df (t_b^k - t_start)) (the DFT of
    Eqs. 19-20 at an arbitrary frequency).  This is the quantity whose
    gradient the adjoint computes."""
    r = resampled_series(x_h, tmpl, gaps, plan)
    tau_b = r["tb"] - plan.t_start
    e = np.exp(-2j * np.pi * _frac(df * tau_b))
    Fa = np.sum(r["wa"] * e)
    Fb = np.sum(r["wb"] * e)
    return float(two_f(Fa, Fb, r["A"], r["B"], r["C"], plan.sigma2))


def single_bin_two_f_many(x_h, tmpl, gaps, plan, dfs):
    """``single_bin_two_f`` at several frequency offsets (series computed once)."""
    r = resampled_series(x_h, tmpl, gaps, plan)
    tau_b = r["tb"] - plan.t_start
    out = np.empty(len(dfs))
    for i, df in enumerate(dfs):
        e = np.exp(-2j * np.pi * _frac(df * tau_b))
        out[i] = two_f(np.sum(r["wa"] * e), np.sum(r["wb"] * e), r["A"], r["B"], r["C"], plan.sigma2)
    return out


def single_bin_gradient(x_h, tmpl, gaps, plan, df, steps=None):
    """d(2F)/d(alpha, delta, f, fdot) of ``single_bin_two_f`` by central
    differences with one Richardson extrapolation (FP64).  Default steps:
    1e-6 rad in alpha and delta, 1e-3/T in f, 1e-3/T^2 in fdot, T the span."""
    T = float(tmpl["span_len"]) * plan.dt
    if steps is None:
        steps = (1e-6, 1e-6, 1e-3 / T, 1e-3 / (T * T))
    tmpl = np.array(tmpl, copy=True)

    def f_at(p):
        t = tmpl.copy()
        t["alpha"], t["delta"], t["fdot"] = p[0], p[1], p[3]
        return single_bin_two_f(x_h, t, gaps, plan, p[2])

    p0 = np.array([float(tmpl["alpha"]), float(tmpl["delta"]), float(df),
                   float(tmpl["fdot"])])
    g = np.zeros(4)
    for i in range(4):
        def d(h):
            e = np.zeros(4)
            e[i] = h
            return (f_at(p0 + e) - f_at(p0 - e)) / (2 * h)
        h = steps[i]
        g[i] = (4.0 * d(h / 2) - d(h)) / 3.0
    return g


def noise_gain(plan, u_frac=None):
    """Expected value of 2F in Gaussian noise for the interpolator: 4 times
    the mean of sum_j w_j^2 over a uniform sub-sample offset (1 for nearest
    neighbour).  Used to check the chi^2_4 mean of sinc runs."""
    if plan.interp == resample.NEAREST:
        return 4.0
    half = plan.taps // 2
    d = np.linspace(0.0, 1.0, 4097)[:-1] + 0.5 / 4096 if u_frac is None else u_frac
    s = np.zeros_like(d)
    for i in range(plan.taps):
        x = d + half - 1 - i
        w = np.sinc(x)
        if plan.window == resample.WIN_LANCZOS:
            w = w * np.sinc(x / half)
        s += w * w
    return 4.0 * float(np.mean(s))
