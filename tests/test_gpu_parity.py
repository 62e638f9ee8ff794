"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerance: max_q |2F_gpu - 2F_oracle| / max(2F_oracle, 4) <= 1e-4 for the
mixed-precision path (FP64 time map and phase at knots, FP32 per sample,
FP32 FFT) against the same-algorithm FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import resample as R

from _gpu import (MODES, NOGAPS, injected_series, oracle_two_f, r15, run_compute, run_resample,
                  tie_margin)

pytestmark = pytest.mark.gpu
TOL = 1e-4


def test_tiny_nearest_neighbour_all_bins():
    """12 h, dt 0.5 s, FFT 2^17, NN, one injection at +0.7 Hz."""
    d = synth.tiny_plan()
    inj = synth.random_injection(synth.SEED_BASE, df=0.7)
    x, info = injected_series(d, synth.SEED_BASE, [inj])
    tm = synth.make_templates(inj.alpha, inj.delta, 0.0, 0, d.n_data)
    assert tie_margin(d, tm[0]) > 1e-6       # the NN decision is unique in FP32 and FP64
    got, rc = run_compute(d, x, tm)
    assert rc == 0
    ref = oracle_two_f(d, x, tm[0])
    assert r15(got[0], ref) <= TOL
    q = int(np.argmax(got[0]))
    assert abs(F.bin_frequencies(d.n_fft, d.dt)[q] - 0.7) < 2.0 / (d.n_fft * d.dt)


@pytest.mark.parametrize("interp", [R.NEAREST, R.SINC])
def test_resample_stage_matches_oracle_series(interp):
    """Steps 1-5: w_a, w_b sample by sample and A, B, C, D."""
    d = synth.PlanDesc(dt=0.5, n_data=40000, n_fft=1 << 16, interp=interp, f_het=150.0,
                       max_templates=3)
    gaps = np.array([[3000, 5000], [20000, 20007], [30000, 33000]], np.int64)
    x, _ = injected_series(d, 7, [synth.random_injection(8, df=0.2)], gaps)
    tm = synth.make_templates([0.3, 2.5, 4.0], [-0.2, 0.9, 0.1], [0.0, -1e-9, -5e-9],
                              [0, 100, 1000], [40000, 39000, 30000], 0, 3)
    (wa, wb, abcd), rc = run_resample(d, x, tm, gaps)
    assert rc == 0
    for i in range(3):
        if interp == R.NEAREST:
            assert tie_margin(d, tm[i]) > 1e-6
        r = F.resampled_series(x.astype(np.complex128), tm[i], gaps, d)
        nb = r["n_b"]
        scale = np.max(np.abs(r["wa"])) + np.max(np.abs(r["wb"]))
        assert np.max(np.abs(wa[i, :nb] - r["wa"])) < 2e-5 * scale
        assert np.max(np.abs(wb[i, :nb] - r["wb"])) < 2e-5 * scale
        assert np.all(wa[i, nb:] == 0) and np.all(wb[i, nb:] == 0)
        A, B, C = r["A"], r["B"], r["C"]
        np.testing.assert_allclose(abcd[i, :3], [A, B, C], rtol=1e-6, atol=1e-6 * (A + B))
        np.testing.assert_allclose(abcd[i, 3], A * B - C * C, rtol=1e-5)


@pytest.mark.parametrize("mode", ["fused", "split"])
def test_sinc_with_gaps_several_templates(mode):
    """3 d of data, FFT 2^19, 8-tap Lanczos sinc, gaps, uneven spans and
    spindowns in one batched launch (resampling fused into the first FFT
    pass, or tiled through memory)."""
    d = synth.PlanDesc(dt=0.5, n_data=3 * 172800 // 2 * 2, n_fft=1 << 19, interp=R.SINC,
                       f_het=300.0, max_templates=6)
    gaps = synth.gap_intervals(d.n_data, 0.1, 7200, 43200 // 2, seed=31)
    injs = [synth.random_injection(40 + i, df=0.05 * (i + 1), fdot=-1e-9 * i) for i in range(2)]
    x, _ = injected_series(d, 41, injs, gaps)
    al = [injs[0].alpha, injs[1].alpha, 1.0, 2.0, 3.0, 5.5]
    de = [injs[0].delta, injs[1].delta, 0.5, -1.2, 0.0, 1.4]
    fd = [injs[0].fdot, injs[1].fdot, -3e-9, 0.0, -1e-8, -2e-10]
    ss = [0, 0, 5000, 0, 20000, 777]
    sl = [d.n_data, d.n_data, 200000, 259200, 150001, 250000]
    tm = synth.make_templates(al, de, fd, ss, sl, 0, len(gaps))
    got, rc = run_compute(d, x, tm, gaps, mode=MODES[mode])
    assert rc == 0
    for i in range(len(tm)):
        ref = oracle_two_f(d, x, tm[i], gaps)
        assert r15(got[i], ref) <= TOL, i


@pytest.mark.parametrize("mode", ["plain", "split"])
@pytest.mark.parametrize("interp", [R.NEAREST, R.SINC])
def test_unfused_and_fused_agree(mode, interp):
    """The tiled resampler + load-mode first pass against the fused pass, at
    a shape whose first-pass block holds several columns (2^17 = 2^9 x 2^8:
    the column tiles and the tile of the resampler differ)."""
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=60000, n_fft=1 << 17, interp=interp, f_het=80.0,
                       max_templates=3)
    x, _ = injected_series(d, 3, [synth.random_injection(4, df=0.3)])
    tm = synth.make_templates([1.0, 2.0, 4.0], [0.3, -0.3, 1.0], [0.0, -2e-9, -1e-8], [0, 0, 999],
                              [d.n_data, d.n_data, 41001])
    a, rc1 = run_compute(d, x, tm, mode=fs.MODE_FUSED)
    b, rc2 = run_compute(d, x, tm, mode=MODES[mode])
    assert rc1 == 0 and rc2 == 0
    assert r15(a, b) < 1e-6
    for i in range(3):
        assert r15(b[i], oracle_two_f(d, x, tm[i])) <= TOL


def test_split_mode_every_factorisation():
    """The tiled resampler and both passes at every first-pass length of a
    2^18 FFT (N1 = 2^6 .. 2^12: columns per block from 16 down to 2, rows
    per second-pass block from 1 up to 16, tile widths from 128 to 256):
    every shape against the oracle, and the shapes against each other."""
    d = synth.PlanDesc(dt=0.5, n_data=120_001, n_fft=1 << 18, interp=R.SINC, f_het=120.0,
                       max_templates=2)
    gaps = synth.gap_intervals(d.n_data, 0.1, 3600, 9000, seed=17)
    x, _ = injected_series(d, 18, [synth.random_injection(19, df=-0.3)], gaps)
    tm = synth.make_templates([0.7, 3.9], [-0.4, 0.9], [-1e-9, 0.0], [0, 1001], [d.n_data, 100_000],
                              0, len(gaps))
    refs = [oracle_two_f(d, x, tm[i], gaps) for i in range(2)]
    outs = []
    for l1 in (6, 8, 10, 12):
        got, rc = run_compute(d, x, tm, gaps, mode=MODES["split"], tuning={"log2_n1": l1})
        assert rc == 0, l1
        for i in range(2):
            assert r15(got[i], refs[i]) <= TOL, (l1, i)
        outs.append(got)
    for got in outs[1:]:
        assert r15(got, outs[0]) < 1e-5


@pytest.mark.parametrize("mode", ["fused", "split"])
def test_fp64_mode_tight(mode):
    """All-FP64 path: agreement with the FP64 oracle to 1e-6 (the floor is the
    cubic interpolation of a, b between knots, ~1e-7, and the float32
    output)."""
    d = synth.PlanDesc(dt=0.5, n_data=50000, n_fft=1 << 16, interp=R.SINC, f_het=1000.0,
                       precision=synth.PREC_FP64, max_templates=2)
    x, _ = injected_series(d, 5, [synth.random_injection(6, df=0.4, fdot=-5e-9)])
    tm = synth.make_templates([0.5, 4.4], [0.7, -0.1], [-5e-9, 0.0], 0, d.n_data)
    got, rc = run_compute(d, x, tm, mode=MODES[mode])
    assert rc == 0
    for i in range(2):
        assert r15(got[i], oracle_two_f(d, x, tm[i])) <= 1e-6


def test_second_spindown_against_oracle():
    """Templates with a second spindown (Eq. 4 to s = 2): the knots carry
    fddot tau^3 / 6 in the phase; 2F in every bin against the oracle, and
    the injection recovered only with its own fddot."""
    d = synth.PlanDesc(dt=0.5, n_data=300_000, n_fft=1 << 19, interp=R.SINC, f_het=110.0,
                       max_templates=3)
    inj = synth.random_injection(81, df=0.2, fdot=-2e-9, fddot=1e-14)   # 5.6 cycles over the span
    x, info = injected_series(d, 82, [inj])
    tm = synth.make_templates([inj.alpha] * 3, inj.delta, inj.fdot, 0, d.n_data,
                              fddot=[inj.fddot, 0.0, -inj.fddot])
    got, rc = run_compute(d, x, tm)
    assert rc == 0
    refs = [oracle_two_f(d, x, tm[i]) for i in range(3)]
    for i in range(3):
        assert r15(got[i], refs[i]) <= TOL, i
    assert np.max(got[0]) > 2 * np.max(got[1])


@pytest.mark.parametrize("mode", ["fused", "split"])
def test_invalid_template_reports_status_and_nan(mode):
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=20000, n_fft=1 << 15, interp=R.NEAREST, max_templates=3)
    x = synth.complex_noise(d.n_data, 1.0, 9)
    tm = synth.make_templates([1.0, 1.0, 1.0], [0.2, 0.2, 0.2], 0.0,
                              [0, 15000, 0], [20000, 10000, 20000])
    got, rc = run_compute(d, x, tm, mode=MODES[mode])
    assert rc == fs._lib.FSTAT_ERANGE
    assert np.all(np.isfinite(got[0])) and np.all(np.isnan(got[1])) and np.all(np.isfinite(got[2]))
    assert r15(got[2], oracle_two_f(d, x, tm[2])) <= TOL


def test_fft_shorter_than_grid_is_range_error():
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=5000, n_fft=1 << 12, interp=R.NEAREST, max_templates=1)
    x = synth.complex_noise(d.n_data, 1.0, 10)
    tm = synth.make_templates(1.0, 0.2, 0.0, 0, 5000)
    got, rc = run_compute(d, x, tm)
    assert rc == fs._lib.FSTAT_ERANGE and np.all(np.isnan(got))


def test_host_grid_length_matches_oracle():
    import paper_0912_4255_gb300 as fs
    from oracle import timemap as TM
    d = synth.search_plan(max_templates=16)
    tm = synth.search_templates(4, 4)
    plan = fs.Plan(d)
    nb = fs.fstat_template_nb(plan, tm)
    for i in range(len(tm)):
        assert nb[i] == TM.grid(tm[i], d)[1]


def test_grid_length_within_velocity_bound():
    """The tiled resampler's grid is sized from n_b <= (n_data - 1)(1 + beta)
    + 1 with beta = (2 pi/year) AU/c + (2 pi/sidereal day) R/c, the largest
    |dt_m/dt| of the analytic ephemeris (Eq. 4pt2).  The host n_b of sky
    positions all over the sphere, those in the ecliptic and at the extremes
    of the orbital Doppler included, stays within it."""
    import paper_0912_4255_gb300 as fs
    d = synth.search_plan(max_templates=16)
    c = 299792458.0
    beta = 2 * np.pi / d.eph.year_s * d.eph.au_m / c + 2 * np.pi / d.eph.sidereal_day_s * d.det.radius_m / c
    bound = (d.n_data - 1) * (1 + beta) + 1
    plan = fs.Plan(d)
    eps = d.eph.obliquity_rad
    lam = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    # ecliptic longitudes -> equatorial (alpha, delta) on the ecliptic
    al = np.arctan2(np.sin(lam) * np.cos(eps), np.cos(lam)) % (2 * np.pi)
    de = np.arcsin(np.sin(lam) * np.sin(eps))
    a2, d2 = synth.fibonacci_sky(192)
    al = np.concatenate([al, a2]); de = np.concatenate([de, d2])
    tm = synth.make_templates(al, de, 0.0, 0, d.n_data)
    nb = fs.fstat_template_nb(plan, tm)
    assert nb.max() <= bound
    # the Doppler of the orbit moves the bound: some position gets close to it
    assert nb.max() > (d.n_data - 1) * (1 + 0.5 * beta)


def test_search_size_full_bins():
    """Search-sized workload (10 d, 1,728,000 samples, FFT 2^22, 10 % gaps,
    8-tap sinc) in the launch configuration the benchmark times: every bin
    of two templates (one at an injection) against the oracle."""
    d = synth.search_plan(max_templates=4)
    gaps = synth.gap_intervals(d.n_data, 0.10, 7200, 43200, seed=synth.SEED_BASE + 1)
    a, dl = synth.fibonacci_sky(1024)
    inj = synth.random_injection(synth.SEED_BASE + 2, df=0.25, fdot=-1e-9 * 3 / 7,
                                 alpha=float(a[100]), delta=float(dl[100]))
    x, info = injected_series(d, synth.SEED_BASE + 1, [inj], gaps)
    tm = synth.make_templates([a[100], a[700], a[3], a[1000]], [dl[100], dl[700], dl[3], dl[1000]],
                              [inj.fdot, -1e-9, 0.0, -5e-10], 0, d.n_data, 0, len(gaps))
    got, rc = run_compute(d, x, tm, gaps)
    assert rc == 0
    for i in (0, 1):
        ref = oracle_two_f(d, x, tm[i], gaps)
        assert r15(got[i], ref) <= TOL, i
    # the other two: sampled bins against direct sums of the resampled series
    fr = F.bin_frequencies(d.n_fft, d.dt)
    rng = synth.rng(5)
    for i in (2, 3):
        q = rng.integers(0, d.n_fft, 24)
        ref = F.single_bin_two_f_many(x.astype(np.complex128), tm[i], gaps, d, fr[q])
        assert r15(got[i][q], ref) <= TOL, i
