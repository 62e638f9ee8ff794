"""Pins of the FP64 oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage or identity it relies on; together
they are chosen so that a dropped term, a wrong sign or index, or a
transposed operand anywhere in ``oracle`` fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import fstat as F
from oracle import geometry as G
from oracle import inject as I
from oracle import resample as R
from oracle import timemap as TM

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")
NOGAPS = np.zeros((0, 2), np.int64)


def facts():
    with open(GOLDEN) as f:
        return json.load(f)


def small_plan(**kw):
    base = dict(dt=0.5, n_data=2048, n_fft=4096, f_het=100.0)
    base.update(kw)
    return synth.PlanDesc(**base)


# ---------------------------------------------------------------- geometry

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_beam_closed_form_is_tensor_form_up_to_orthogonal_map(seed):
    """Eqs. 2-3: a, b from the JKS closed form and from d:eps_+, d:eps_x must
    be related by one constant orthogonal 2x2 map (a change of polarisation
    basis).  A wrong coefficient makes the map time-dependent or
    non-orthogonal."""
    g = synth.rng(seed)
    det = synth.Detector(lat_rad=g.uniform(-1.4, 1.4), lon_rad=g.uniform(-3, 3),
                         gamma_rad=g.uniform(0, math.pi))
    plan = synth.PlanDesc(det=det)
    alpha, delta = g.uniform(0, 2 * math.pi), math.asin(g.uniform(-1, 1))
    t = np.linspace(0, 3 * 86400, 3001)
    a, b = G.beam_ab(t, alpha, delta, plan.det, plan.eph)
    fp, fx = G.antenna_tensor(t, alpha, delta, 0.0, plan.det, plan.eph)
    X = np.stack([a, b], 1)
    Y = np.stack([fp, fx], 1)
    M, *_ = np.linalg.lstsq(X, Y, rcond=None)
    assert np.max(np.abs(X @ M - Y)) < 1e-12
    assert np.allclose(M.T @ M, np.eye(2), atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_antenna_functions_follow_eqs_2_3(seed):
    """Eqs. 2-3 with zeta = 90 deg: F_+ = a cos 2psi + b sin 2psi and
    F_x = b cos 2psi - a sin 2psi, the tensor contraction against the JKS
    closed form at several polarisation angles (a flipped sign of eps_x or of
    psi fails here)."""
    g = synth.rng(seed)
    det = synth.Detector(lat_rad=g.uniform(-1.4, 1.4), lon_rad=g.uniform(-3, 3),
                         gamma_rad=g.uniform(0, math.pi))
    plan = synth.PlanDesc(det=det)
    alpha, delta = g.uniform(0, 2 * math.pi), math.asin(g.uniform(-1, 1))
    t = np.linspace(0, 86400, 501)
    a, b = G.beam_ab(t, alpha, delta, plan.det, plan.eph)
    for psi in (0.0, 0.3, 1.2, 2.9):
        c, s = math.cos(2 * psi), math.sin(2 * psi)
        fp, fx = G.antenna_tensor(t, alpha, delta, psi, plan.det, plan.eph)
        assert np.max(np.abs(fp - (a * c + b * s))) < 1e-12
        assert np.max(np.abs(fx - (b * c - a * s))) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sky_average_of_beam_power_is_two_fifths(seed):
    """Eqs. 2-3 give F_+^2 + F_x^2 = a^2 + b^2 (zeta = 90 deg) at every
    polarisation angle, and the average of F_+^2 + F_x^2 of an interferometer
    with perpendicular arms over an isotropic sky is the textbook 2/5, for
    any latitude and arm orientation.  A wrong coefficient in the closed form
    of a, b (one that the orthogonal-map pin above cannot see, e.g. a common
    scale) breaks it.  The sky and one sidereal day are sampled exactly for
    the harmonics involved."""
    g = synth.rng(40 + seed)
    det = synth.Detector(lat_rad=g.uniform(-1.4, 1.4), lon_rad=g.uniform(-3, 3),
                         gamma_rad=g.uniform(0, math.pi))
    plan = synth.PlanDesc(det=det)
    alpha, delta = synth.fibonacci_sky(4096)
    t = np.linspace(0.0, plan.eph.sidereal_day_s, 16, endpoint=False)
    tot = cross = 0.0
    for al, de in zip(alpha, delta):
        a, b = G.beam_ab(t, al, de, plan.det, plan.eph)[:2]
        tot += np.mean(a * a + b * b)
        cross += np.mean(a * b)
    assert abs(tot / len(alpha) - 0.4) < 1e-5
    assert abs(cross / len(alpha)) < 1e-6


def test_beam_zenith_unit_response():
    """Sec. II after Eq. 3 (zeta = 90 deg): for a source at the zenith the
    response to an optimally oriented wave is 1, i.e. a^2 + b^2 = 1."""
    assert facts()["arm_angle_deg"]["zeta"] == 90.0
    plan = synth.PlanDesc()
    t = 12345.0
    theta = float(G.sidereal_angle(t, plan.eph, plan.det))
    a, b = G.beam_ab(t, theta, plan.det.lat_rad, plan.det, plan.eph)
    assert abs(a * a + b * b - 1.0) < 1e-13


def test_roemer_delay_magnitudes_and_rate():
    """Eq. 4pt2 and Eq. 11c with the analytic ephemeris: |t_m| <= (AU + R)/c,
    the orbital amplitude is AU/c = 499.005 s for a source in the ecliptic,
    the Doppler factor is of order 1e-4 (text after Eq. 11c) and is the time
    derivative of t_m."""
    plan = synth.PlanDesc()
    f = facts()["max_doppler"]
    t = np.linspace(0, plan.eph.year_s, 20001)
    # ecliptic pole direction has no orbital term; ecliptic source has it all
    eps = plan.eph.obliquity_rad
    a_ecl, d_ecl = 0.0, 0.0     # vernal equinox lies in the ecliptic
    tm = G.roemer_delay(t, a_ecl, d_ecl, plan.det, plan.eph)
    au_c = plan.eph.au_m / G.C_LIGHT
    r_c = plan.det.radius_m / G.C_LIGHT
    assert abs(au_c - 499.00478) < 1e-4
    assert np.max(np.abs(tm)) <= au_c + r_c + 1e-9
    assert np.max(tm) > au_c - r_c - 1e-3
    rate = G.roemer_rate(t, a_ecl, d_ecl, plan.det, plan.eph)
    assert 0.5 * f["order"] < np.max(np.abs(rate)) < 2 * f["order"]
    h = 1.0
    fd = (G.roemer_delay(t + h, a_ecl, d_ecl, plan.det, plan.eph)
          - G.roemer_delay(t - h, a_ecl, d_ecl, plan.det, plan.eph)) / (2 * h)
    assert np.max(np.abs(fd - rate)) < 1e-12
    # ecliptic pole: only the diurnal term of amplitude R cos(lat)/c survives
    ap, dp = -math.pi / 2, math.pi / 2 - eps
    tmp = G.roemer_delay(t[:2000], ap, dp, plan.det, plan.eph)
    assert np.max(np.abs(tmp)) < r_c + 1e-9


def test_inverse_map_residual():
    """Eq. 21 inverted by fixed-point iteration: T^k + t_m(T^k) = t_b^k."""
    plan = synth.search_plan()
    tm = synth.make_templates(1.3, -0.4, 0.0, 0, plan.n_data)[0]
    tb, T, n_b = TM.resample_times(tm, plan)
    res = T + G.roemer_delay(T, 1.3, -0.4, plan.det, plan.eph) - tb
    assert np.max(np.abs(res)) < 1e-9
    # grid: t_b^k uniform, and the last point within dt of t_b(t_e)
    t_s, t_e = TM.span_times(tm, plan)
    tbe = t_e + float(G.roemer_delay(t_e, 1.3, -0.4, plan.det, plan.eph))
    assert tb[-1] <= tbe + 1e-9 and tb[-1] > tbe - plan.dt
    assert abs(n_b - plan.n_data) < 2 * 1e-4 * plan.n_data


# ---------------------------------------------------------------- heterodyne / injection model

def test_heterodyne_worked_example():
    """Sec. III.A.1 worked example: heterodyning at 995 Hz moves 990 Hz to
    -5 Hz and 1000 Hz to +5 Hz; keeping every 100th point of the 1 kHz-rate
    stream gives 10 Hz sampling.  The oracle's reading x_h = x e^{-2 pi i f_h t}
    must reproduce it."""
    ex = facts()["heterodyne_example"]
    fs = 1000.0 * 8                      # well above 2 kHz
    t = np.arange(int(fs * 20)) / fs
    for f_in, f_out in [(ex["band_hz"][1], ex["high_edge_after_hz"]),
                        (ex["band_hz"][0], ex["low_edge_after_hz"])]:
        x = np.exp(2j * np.pi * f_in * t)          # analytic tone
        xh = x * np.exp(-2j * np.pi * ex["f_het_hz"] * t)
        spec = np.fft.fftshift(np.fft.fft(xh))
        fr = np.fft.fftshift(np.fft.fftfreq(t.size, 1 / fs))
        assert abs(fr[np.argmax(np.abs(spec))] - f_out) < 1e-9
    assert fs / 8 / ex["decimation"] == ex["sample_rate_after_hz"]


def test_injection_is_positive_frequency_half_of_real_strain():
    """Eq. 1 with h_+ = A_+ cos Psi, h_x = A_x sin Psi: demodulating the real
    strain by its own phase over many cycles leaves the complex amplitude
    (F_+ A_+ - i F_x A_x)/2 that ``inject.signal`` uses."""
    plan = synth.PlanDesc(f_het=995.0, dt=0.5)
    inj = synth.random_injection(7, df=0.7, fdot=0.0)
    h0 = 1.0
    fs = 16000.0
    t0 = 4321.0
    t = t0 + np.arange(int(fs * 2.0)) / fs
    tm = G.roemer_delay(t, inj.alpha, inj.delta, plan.det, plan.eph)
    tau = t - plan.t_start + tm
    psi = inj.phi0 + 2 * np.pi * (plan.f_het + inj.df) * tau
    Fp, Fx = G.antenna_tensor(t, inj.alpha, inj.delta, inj.psi, plan.det, plan.eph)
    Ap, Ax = h0 * (1 + inj.cosi ** 2) / 2, h0 * inj.cosi
    h = Fp * Ap * np.cos(psi) + Fx * Ax * np.sin(psi)
    amp = np.mean(h * np.exp(-1j * psi))
    # inject.signal at the window's midpoint, divided by its own phase factor
    tt = t0 + 1.0
    p1 = synth.PlanDesc(f_het=995.0, dt=1.0 / fs, t_start=tt, n_data=1,
                        det=plan.det, eph=plan.eph)
    s = I.signal(inj, p1, n_data=1, h0=h0)[0]
    tmm = float(G.roemer_delay(tt, inj.alpha, inj.delta, plan.det, plan.eph))
    # with t_start = tt: tau = t_m, and x_h's phase is Phi_0 + 2 pi (f_h + df) t_m
    amp_inj = s / np.exp(1j * (inj.phi0 + 2 * np.pi * (p1.f_het + inj.df) * tmm))
    assert abs(amp - amp_inj) < 2e-4 * max(abs(amp), 1e-3)


# ---------------------------------------------------------------- resampling pieces

def test_sinc_interpolator_tap_positions():
    """Truncated windowed sinc on a slowly varying tone reproduces the tone
    (a tap shifted by one sample would be off by ~30 %)."""
    n = 400
    j = np.arange(n)
    nu = 0.03
    x = np.exp(2j * np.pi * nu * j)
    u = np.linspace(10.0, 380.0, 1777)
    valid = np.ones(n, bool)
    # Lanczos is accurate to ~3e-3 here; plain truncation has the ~6 %
    # ripple of a truncated Dirichlet kernel; a one-sample shift errs by ~0.19
    for window, tol in ((R.WIN_LANCZOS, 5e-3), (R.WIN_RECT, 8e-2)):
        z = R.interpolate(x, u, valid, R.SINC, 8, window)
        assert np.max(np.abs(z - np.exp(2j * np.pi * nu * u))) < tol
    # at integer positions the interpolator returns the sample itself
    z = R.interpolate(x, np.arange(20.0, 30.0), valid, R.SINC, 8, R.WIN_LANCZOS)
    assert np.allclose(z, x[20:30], atol=1e-15)
    zn = R.interpolate(x, np.array([20.49, 20.51]), valid, R.NEAREST)
    assert zn[0] == x[20] and zn[1] == x[21]


def test_gap_taps_and_mask():
    """Sec. III.B, gaps: samples in a gap contribute nothing; the mask
    follows the nearest-neighbour source."""
    n = 100
    x = np.ones(n, np.complex128)
    valid = R.valid_samples(n, 5, 90, np.array([[40, 50]]))
    assert valid[5] and not valid[4] and not valid[40] and valid[50] and not valid[95]
    u = np.array([39.4, 39.6, 49.4, 49.6, 4.4, 4.6])
    m = R.mask(u, valid)
    assert list(m) == [1, 0, 0, 1, 0, 1]
    z = R.interpolate(x, np.array([45.0]), valid, R.SINC, 8, R.WIN_LANCZOS)
    assert abs(z[0]) < 1e-15


# ---------------------------------------------------------------- F-statistic

def _brute_force_two_f(r, plan, n_fft):
    k = np.arange(r["n_b"])
    q = np.arange(n_fft)
    df = (q - n_fft // 2) / (n_fft * plan.dt)
    E = np.exp(-2j * np.pi * np.outer(df, k * plan.dt))
    Fa = E @ r["wa"]
    Fb = E @ r["wb"]
    return F.two_f(Fa, Fb, r["A"], r["B"], r["C"], plan.sigma2)


@pytest.mark.parametrize("interp", [R.NEAREST, R.SINC])
def test_fft_matches_brute_force_dft(interp):
    """Step 6 (Eqs. 19-20): the FFT of the zero-padded weighted series with
    the ascending-frequency reordering equals an O(N^2) DFT evaluated at
    df_q = (q - N/2)/(N dt)."""
    plan = synth.PlanDesc(dt=0.5, n_data=200, n_fft=256, interp=interp, f_het=37.0)
    x = synth.complex_noise(plan.n_data, 1.0, 11)
    tm = synth.make_templates(2.0, 0.3, -1e-7, 3, 190)[0]
    r = F.resample_two_f(x, tm, NOGAPS, plan, return_parts=True)
    bf = _brute_force_two_f(r, plan, plan.n_fft)
    assert np.max(np.abs(r["two_f"] - bf)) < 1e-9 * max(1.0, np.max(bf))


@pytest.mark.parametrize("interp", [R.NEAREST, R.SINC])
def test_zero_ephemeris_resampling_equals_direct(interp):
    """With AU = R = 0 the Roemer delay vanishes, T^k = t_b^k falls on the
    data grid, interpolation is exact, and the resampling 2F must equal direct
    demodulation (Eqs. 7-8) at every FFT bin, gaps included."""
    eph = synth.Ephem(au_m=0.0)
    det = synth.Detector(radius_m=0.0)
    plan = synth.PlanDesc(dt=0.5, n_data=3000, n_fft=4096, interp=interp,
                          f_het=50.0, det=det, eph=eph)
    x = synth.complex_noise(plan.n_data, 1.0, 5)
    gaps = np.array([[400, 650], [1700, 1800]], np.int64)
    x = synth.zero_gaps(x, gaps)
    tm = synth.make_templates(0.7, 0.2, -3e-8, 10, 2900, 0, 2)[0]
    r = F.resample_two_f(x, tm, gaps, plan, return_parts=True)
    assert r["n_b"] == 2900
    fr = F.bin_frequencies(plan.n_fft, plan.dt)
    sel = np.arange(0, plan.n_fft, 37)
    d = F.direct_two_f(x, tm, gaps, plan, fr[sel])
    assert np.max(np.abs(r["two_f"][sel] - d)) < 1e-9 * np.max(d)


@pytest.mark.parametrize("seed,fdot,f_het", [(1, 0.0, 100.0), (2, -1e-8, 1000.0),
                                              (3, -3e-9, 400.0)])
def test_noise_free_direct_demod_gives_rho2(seed, fdot, f_het):
    """Eq. 6 with Eqs. 7-10: for noise-free data at the true template the
    maximised statistic recovers all signal power, 2F = rho^2 (the
    non-centrality of Sec. IV.B), gaps included."""
    plan = synth.PlanDesc(dt=0.5, n_data=40000, f_het=f_het)
    gaps = np.array([[5000, 9000], [20000, 21000]], np.int64)
    valid = I.valid_all(plan, gaps)
    inj = synth.random_injection(seed, df=0.31, fdot=fdot)
    x, info = I.inject(np.zeros(plan.n_data), [inj], plan, valid)
    tm = synth.make_templates(inj.alpha, inj.delta, fdot, 0, plan.n_data, 0, 2)[0]
    d = F.direct_two_f(x, tm, gaps, plan, [inj.df])[0]
    assert abs(d - info[0][1]) < 1e-9 * info[0][1]
    assert abs(info[0][1] - 400.0) < 1e-9


def test_spindown_and_heterodyne_signs():
    """Eq. 7 with Eq. 5 (demodulate by exp(-i Phi_s)) and the 995 Hz example
    (x_h = x exp(-2 pi i f_h t)): the true signs recover rho^2; flipping the
    spindown loses most of it, and the resampled peak lands at +df."""
    plan = synth.PlanDesc(dt=0.5, n_data=86400, n_fft=1 << 17, f_het=200.0,
                          interp=R.SINC)
    valid = I.valid_all(plan)
    df = 2000 / (plan.n_fft * plan.dt)          # on-grid, +0.0305 Hz
    inj = synth.random_injection(4, df=df, fdot=-2e-8)
    x, info = I.inject(np.zeros(plan.n_data), [inj], plan, valid)
    good = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, plan.n_data)[0]
    bad = synth.make_templates(inj.alpha, inj.delta, -inj.fdot, 0, plan.n_data)[0]
    r = F.resample_two_f(x, good, NOGAPS, plan)
    rb = F.resample_two_f(x, bad, NOGAPS, plan)
    q = int(np.argmax(r))
    assert q == plan.n_fft // 2 + 2000
    assert r[q] > 0.98 * info[0][1]
    assert np.max(rb) < 0.2 * info[0][1]


def test_second_spindown_phase():
    """Eq. 4 to s = 2: a signal with a second spindown is recovered to
    rho^2 (noise-free direct demodulation) only by the template with the
    same fddot; without it, or with the opposite sign, the phase runs
    ~10 cycles off over the span and the power is lost."""
    plan = synth.PlanDesc(dt=0.5, n_data=4 * 86400 * 2, n_fft=1 << 20, f_het=150.0, interp=R.SINC)
    valid = I.valid_all(plan)
    inj = synth.random_injection(14, df=0.125, fdot=-3e-10, fddot=4e-16)
    x, info = I.inject(np.zeros(plan.n_data), [inj], plan, valid)
    rho2 = info[0][1]
    got = {}
    for name, fdd in (("same", inj.fddot), ("none", 0.0), ("flip", -inj.fddot)):
        t = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, plan.n_data, fddot=fdd)[0]
        got[name] = float(F.direct_two_f(x, t, NOGAPS, plan, inj.df)[0])
    assert abs(got["same"] - rho2) / rho2 < 1e-9
    assert got["none"] < 0.3 * rho2 and got["flip"] < 0.3 * rho2


def test_nearest_neighbour_loss_is_sinc_squared():
    """Sec. V.B: interpolation loses power towards the band edge (of order
    30 %).  For nearest-neighbour resampling with rounding errors spread
    uniformly over a sample the expected power factor at df is
    sinc^2(df dt); at df = 0.7 Hz, dt = 0.5 s this is 0.657."""
    fct = facts()["interpolation_loss"]
    plan = synth.PlanDesc(dt=0.5, n_data=10 * 86400 * 2 // 4, n_fft=1 << 19,
                          interp=R.NEAREST, f_het=100.0)
    valid = I.valid_all(plan)
    k = round(0.7 * plan.n_fft * plan.dt)
    df = k / (plan.n_fft * plan.dt)
    ratios = []
    for seed in (21, 22, 23):
        inj = synth.random_injection(seed, df=df)
        x, info = I.inject(np.zeros(plan.n_data), [inj], plan, valid)
        tm = synth.make_templates(inj.alpha, inj.delta, 0.0, 0, plan.n_data)[0]
        r = F.resample_two_f(x, tm, NOGAPS, plan)
        ratios.append(r[plan.n_fft // 2 + k] / info[0][1])
    expect = np.sinc(df * plan.dt) ** 2
    assert abs(np.mean(ratios) - expect) < 0.05
    assert abs((1 - expect) - fct["order"]) < 0.1


def test_doubling_the_band_follows_the_sinc_squared_law():
    """Sec. V.B's remedy, nearest neighbour: the same signal in data
    sampled twice as fast (dt / 2, twice the band) loses only
    1 - sinc^2(df dt / 2) of its power, and the signal's bin then lies in
    the central half of the doubled band, the half that is kept."""
    ratios = []
    for seed in (24, 25, 26):
        plan = synth.PlanDesc(dt=0.25, n_data=5 * 86400 * 2, n_fft=1 << 20, interp=R.NEAREST,
                              f_het=100.0)
        k = round(0.7 * plan.n_fft * plan.dt)
        df = k / (plan.n_fft * plan.dt)
        assert plan.n_fft // 4 <= plan.n_fft // 2 + k < 3 * plan.n_fft // 4
        inj = synth.random_injection(seed, df=df)
        x, info = I.inject(np.zeros(plan.n_data), [inj], plan, I.valid_all(plan))
        tm = synth.make_templates(inj.alpha, inj.delta, 0.0, 0, plan.n_data)[0]
        r = F.resample_two_f(x, tm, NOGAPS, plan)
        ratios.append(r[plan.n_fft // 2 + k] / info[0][1])
    expect = np.sinc(df * plan.dt) ** 2               # 0.903 at 0.7 Hz, against 0.657 at dt = 0.5 s
    assert abs(np.mean(ratios) - expect) < 0.03
    assert np.mean(ratios) > np.sinc(df * 0.5) ** 2 + 0.2


def test_chi2_four_dof_in_noise():
    """Sec. IV.B: in Gaussian noise 2F is chi^2 with 4 degrees of freedom
    (mean 4, variance 8), here through the whole resampling path."""
    dof = facts()["chi2_dof"]["dof"]
    plan = small_plan(n_data=1024, n_fft=2048, interp=R.NEAREST)
    tm = synth.make_templates(1.1, 0.5, 0.0, 0, plan.n_data)[0]
    vals = []
    for s in range(600):
        x = synth.complex_noise(plan.n_data, plan.sigma2, 1000 + s)
        r = F.resample_two_f(x, tm, NOGAPS, plan)
        vals.extend(r[[100, 700, 1300, 1900]])
    vals = np.asarray(vals)
    assert abs(vals.mean() - dof) < 0.15
    assert abs(vals.var() - 2 * dof) < 1.2
    assert stats.kstest(vals, "chi2", args=(dof,)).pvalue > 1e-3


def test_sinc_noise_mean_matches_tap_energy():
    """Parseval: for sinc resampling the mean of 2F over all bins in noise is
    4 times the mean tap energy sum_j w_j^2."""
    plan = small_plan(n_data=8192, n_fft=16384, interp=R.SINC, window=R.WIN_LANCZOS)
    tm = synth.make_templates(1.1, 0.5, 0.0, 0, plan.n_data)[0]
    m = []
    for s in range(4):
        x = synth.complex_noise(plan.n_data, plan.sigma2, 50 + s)
        m.append(np.mean(F.resample_two_f(x, tm, NOGAPS, plan)))
    assert abs(np.mean(m) / F.noise_gain(plan) - 1.0) < 0.03


def test_single_bin_form_matches_fft_bin():
    """The single-bin DFT used for the gradient equals the FFT path at an
    FFT bin frequency (the grid-start phase is common to F_a and F_b)."""
    plan = small_plan(n_data=3000, n_fft=4096, interp=R.SINC)
    x = synth.complex_noise(plan.n_data, 1.0, 9)
    tm = synth.make_templates(0.4, -0.9, -2e-9, 0, plan.n_data)[0]
    r = F.resample_two_f(x, tm, NOGAPS, plan)
    fr = F.bin_frequencies(plan.n_fft, plan.dt)
    for q in (0, 17, 2048, 3001):
        assert abs(F.single_bin_two_f(x, tm, NOGAPS, plan, fr[q]) - r[q]) < 1e-9 * max(r[q], 1)


def test_single_bin_many_matches_single_bin_and_fft_bins():
    """``single_bin_two_f_many`` (the sampled-bin reference of the full-size
    parity tests) is ``single_bin_two_f`` evaluated at several offsets: equal
    to it at off-grid frequencies, and equal to the FFT path (itself pinned
    by brute-force DFT) at bin frequencies.  A wrong sign or scale of the
    frequency fails (a shift of the phase reference does not change 2F)."""
    plan = small_plan(n_data=3000, n_fft=4096, interp=R.SINC)
    x = synth.complex_noise(plan.n_data, 1.0, 19)
    inj = synth.random_injection(23, df=0.27, fdot=-2e-9)
    x = x + I.inject(np.zeros(plan.n_data, np.complex128), [inj], plan,
                     np.ones(plan.n_data, bool))[0]
    tm = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, plan.n_data)[0]
    r = F.resample_two_f(x, tm, NOGAPS, plan)
    fr = F.bin_frequencies(plan.n_fft, plan.dt)
    qs = [0, 17, 2048, int(np.argmax(r)), 3001, 4095]
    many = F.single_bin_two_f_many(x, tm, NOGAPS, plan, fr[qs])
    for q, v in zip(qs, many):
        assert abs(v - r[q]) < 1e-9 * max(r[q], 1)
    offs = [0.27, -0.3112, 0.0001, 0.9]
    many = F.single_bin_two_f_many(x, tm, NOGAPS, plan, offs)
    for f, v in zip(offs, many):
        one = F.single_bin_two_f(x, tm, NOGAPS, plan, f)
        assert abs(v - one) < 1e-12 * max(one, 1)
    assert many[0] > 50 * np.median(r)                 # the injection is where it belongs


def test_gradient_analytic_in_f_and_fdot():
    """d2F/df and d2F/dfdot have closed forms from dF_a/df = sum w_a
    (-2 pi i tau) e and dw/dfdot = -i pi tau^2 w; the finite-difference
    gradient must agree."""
    plan = small_plan(n_data=6000, n_fft=8192, interp=R.SINC)
    x = synth.complex_noise(plan.n_data, 1.0, 77)
    tm = synth.make_templates(2.2, 0.1, -1e-8, 0, plan.n_data)[0]
    df = 0.123
    r = F.resampled_series(x, tm, NOGAPS, plan)
    tb = r["tb"] - plan.t_start
    e = np.exp(-2j * np.pi * df * tb)
    Fa, Fb = np.sum(r["wa"] * e), np.sum(r["wb"] * e)
    A, B, C = r["A"], r["B"], r["C"]
    D = A * B - C * C

    def d2f(dFa, dFb):
        return 2 * (2 * B * np.real(np.conj(Fa) * dFa) + 2 * A * np.real(np.conj(Fb) * dFb)
                    - 2 * C * np.real(dFa * np.conj(Fb) + Fa * np.conj(dFb))) / (plan.sigma2 * D)

    g_f = d2f(np.sum(r["wa"] * e * (-2j * np.pi * tb)), np.sum(r["wb"] * e * (-2j * np.pi * tb)))
    g_fd = d2f(np.sum(r["wa"] * e * (-1j * np.pi * tb * tb)),
               np.sum(r["wb"] * e * (-1j * np.pi * tb * tb)))
    g = F.single_bin_gradient(x, tm, NOGAPS, plan, df)
    assert abs(g[2] - g_f) < 1e-6 * abs(g_f)
    assert abs(g[3] - g_fd) < 1e-5 * abs(g_fd)


def test_gradient_vanishes_at_noise_free_truth():
    """At the true parameters of a noise-free signal 2F is maximal (2F <= rho^2
    by Cauchy-Schwarz, Eq. 6), so the gradient of the direct statistic is
    zero; the resampled single-bin statistic inherits it up to the small
    interpolation error at low df."""
    plan = synth.PlanDesc(dt=0.5, n_data=40000, n_fft=1 << 16, interp=R.SINC, f_het=100.0)
    valid = I.valid_all(plan)
    inj = synth.random_injection(12, df=0.02, fdot=-1e-9)
    x, info = I.inject(np.zeros(plan.n_data), [inj], plan, valid)
    tm = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, plan.n_data)[0]
    T = plan.n_data * plan.dt
    g = F.single_bin_gradient(x, tm, NOGAPS, plan, inj.df)
    # first-order change over one metric scale must be tiny against rho^2
    scale = np.array([1e-3, 1e-3, 1.0 / T, 1.0 / T ** 2])
    assert np.all(np.abs(g * scale) < 2e-3 * info[0][1])
    # away from the truth the gradient points uphill
    tm2 = tm.copy()
    tm2["alpha"] += 2e-3
    g2 = F.single_bin_gradient(x, tm2, NOGAPS, plan, inj.df + 0.3 / T)
    f0 = F.single_bin_two_f(x, tm2, NOGAPS, plan, inj.df + 0.3 / T)
    step = 1e-3 * scale ** 2 * g2 / np.max(np.abs(g2 * scale))
    tm3 = tm2.copy()
    tm3["alpha"] += step[0]
    tm3["delta"] += step[1]
    tm3["fdot"] += step[3]
    f1 = F.single_bin_two_f(x, tm3, NOGAPS, plan, inj.df + 0.3 / T + step[2])
    assert f1 > f0


# ---------------------------------------------------------------- inputs

def test_gap_generator():
    gaps = synth.gap_intervals(100000, 0.1, 2000, 12000, seed=3)
    assert gaps.shape[1] == 2
    assert np.all(gaps[:, 1] > gaps[:, 0])
    assert np.all(gaps[1:, 0] > gaps[:-1, 1])
    cov = int(np.sum(gaps[:, 1] - gaps[:, 0]))
    assert 10000 <= cov < 10000 + 12000
    assert gaps[0, 0] >= 1 and gaps[-1, 1] <= 99999


def test_fibonacci_sky_uniform():
    a, d = synth.fibonacci_sky(4096)
    assert abs(np.mean(np.sin(d))) < 1e-3
    assert np.all((a >= 0) & (a < 2 * math.pi))


# --------------------------------------------------------------- candidates

def test_band_top_k_against_brute_force():
    """Per-band top-k (the step after Eq. 6 that a search applies): brute
    force on small rows with ties and NaN bins."""
    from oracle import candidates as CA
    g = np.random.default_rng(11)
    a = g.integers(0, 6, size=(3, 48)).astype(np.float64)     # many ties
    a[1, 5] = np.nan
    a[2, 16:32] = np.nan                                        # a band with no finite value
    vals, bins = CA.band_top_k(a, 16, 5)
    for r in range(3):
        for b in range(3):
            cand = [(a[r, j], j) for j in range(b * 16, (b + 1) * 16) if not np.isnan(a[r, j])]
            cand.sort(key=lambda t: (-t[0], t[1]))               # largest first, then lower bin
            want = cand[:5] + [(-np.inf, -1)] * (5 - len(cand[:5]))
            assert [tuple(x) for x in zip(vals[r, b], bins[r, b])] == want


def test_band_top_k_is_a_selection():
    """Invariants: descending values, bins inside their band, the values are
    the spectrum's at those bins, and nothing outside exceeds the k-th."""
    from oracle import candidates as CA
    g = np.random.default_rng(12)
    a = g.chisquare(4, size=(2, 4096))
    a[0, 1234] = 90.0
    vals, bins = CA.band_top_k(a, 1024, 8)
    assert np.all(np.diff(vals, axis=2) <= 0)
    for r in range(2):
        for b in range(4):
            assert np.all((bins[r, b] >= b * 1024) & (bins[r, b] < (b + 1) * 1024))
            assert np.array_equal(a[r, bins[r, b]], vals[r, b])
            rest = np.delete(a[r, b * 1024:(b + 1) * 1024], bins[r, b] - b * 1024)
            assert rest.max() <= vals[r, b, -1]
    assert bins[0, 1, 0] == 1234 and vals[0, 1, 0] == 90.0


def test_span_inside_a_gap_has_no_statistic():
    """A template whose whole span lies inside a gap: the mask m is zero on
    the grid (no valid source sample), so A = B = C = 0 and D = 0 (Eqs.
    9-10 as sums over the valid samples), the weighted series are zero, and
    2F (Eq. 6) has no finite value.  A span that overlaps the gap by part
    keeps D > 0 and a finite 2F."""
    desc = synth.tiny_plan(interp=synth.SINC, taps=8)
    gaps = np.array([[10000, 30000]], np.int64)
    x = synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + 97).astype(np.complex128)
    tm = synth.make_templates([1.0, 1.0], [0.3, 0.3], [0.0, 0.0], 0, desc.n_data, 0, 1)
    tm["span_start"] = [12000, 25000]
    tm["span_len"] = [5000, 10000]              # inside the gap; half inside
    r = F.resampled_series(x, tm[0], gaps, desc)
    assert r["A"] == r["B"] == r["C"] == 0.0
    assert not np.any(r["m"]) and not np.any(r["wa"]) and not np.any(r["wb"])
    with np.errstate(divide="ignore", invalid="ignore"):
        assert not np.any(np.isfinite(F.resample_two_f(x, tm[0], gaps, desc)))
    r = F.resampled_series(x, tm[1], gaps, desc)
    assert r["A"] * r["B"] - r["C"] ** 2 > 0.0
    assert 0.4 < np.mean(r["m"]) < 0.6
    assert np.all(np.isfinite(F.resample_two_f(x, tm[1], gaps, desc)))


def test_two_f_invariances():
    """Eq. 6 is a quadratic form F^H M^-1 F with M = [[A, C], [C, B]]: it
    is unchanged by a common phase of the data, by scaling the data and
    sigma^2 together, and by an orthogonal mixing of (a, b) (which mixes
    F_a, F_b and transforms A, B, C as M -> R M R^T).  A wrong sign of the
    cross term, or A and B swapped in it, fails the last check."""
    g = synth.rng(77)
    Fa = g.normal(size=64) + 1j * g.normal(size=64)
    Fb = g.normal(size=64) + 1j * g.normal(size=64)
    A, B, C = 3.0, 2.0, 0.7
    ref = F.two_f(Fa, Fb, A, B, C, 1.0)
    ph = np.exp(1j * 0.83)
    assert np.allclose(F.two_f(Fa * ph, Fb * ph, A, B, C, 1.0), ref, rtol=1e-13, atol=0)
    assert np.allclose(F.two_f(3.0 * Fa, 3.0 * Fb, A, B, C, 9.0), ref, rtol=1e-13, atol=0)
    th = 0.61
    c, s = np.cos(th), np.sin(th)
    rot = np.array([[c, s], [-s, c]])
    M2 = rot @ np.array([[A, C], [C, B]]) @ rot.T
    Fa2, Fb2 = c * Fa + s * Fb, -s * Fa + c * Fb
    assert np.allclose(F.two_f(Fa2, Fb2, M2[0, 0], M2[1, 1], M2[0, 1], 1.0), ref, rtol=1e-12, atol=0)
    # the same through the whole oracle: a sky template's 2F does not change
    # when the data carry a common phase
    d = synth.tiny_plan(n_data=4000, n_fft=1 << 13, interp=R.SINC, taps=8)
    x = synth.complex_noise(d.n_data, d.sigma2, 78).astype(np.complex128)
    tm = synth.make_templates([1.1], [0.4], [0.0], 0, d.n_data)
    a = F.resample_two_f(x, tm[0], np.zeros((0, 2), np.int64), d)
    b = F.resample_two_f(x * ph, tm[0], np.zeros((0, 2), np.int64), d)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-12)
