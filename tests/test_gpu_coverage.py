"""Parity at the configurations the library offers or the benchmark times,
beyond the default shapes of test_gpu_parity.py:

* the search-sized workload at the benchmark's own launch shape (64
  templates per call and per internal launch, an 8 GiB workspace whose
  per-template offsets pass 2^32 bytes);
* every interpolator the ABI accepts: the plain truncated sinc (RECT, the
  interpolator of Sec. III.A.2 step 4) and the Lanczos window at every even
  tap count 2..16 (the 8-tap count has its own compiled path, the others
  the generic one);
* the ragged batch workload at its stated spans of 1, 5 and 10 days (FFT
  lengths 2^18 .. 2^21) through RaggedBatch and a CUDA graph.

Tolerance as elsewhere: R15 <= 1e-4 against the FP64 oracle of the same
algorithm."""
import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import resample as R

from _gpu import MODES, injected_series, oracle_two_f, r15, run_compute

pytestmark = pytest.mark.gpu
TOL = 1e-4


def test_search_size_at_the_benchmark_launch_shape():
    """10 d, 1,728,000 samples, FFT 2^22, 10 % gaps, 8-tap Lanczos; one call
    of 64 consecutive templates of the 8192-template grid, as the benchmark
    makes it (one internal chunk of 64).  Every bin of three templates (the
    first, the last and one at an injection), sampled bins of eight more."""
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.search_plan(max_templates=64)
    gaps = synth.gap_intervals(d.n_data, 0.10, 7200, 43200, seed=synth.SEED_BASE + 1)
    a, dl = synth.fibonacci_sky(1024)
    fd = np.linspace(-1e-9, 0.0, 8)
    tm_all = synth.make_templates(np.repeat(a, 8), np.repeat(dl, 8), np.tile(fd, 1024), 0, d.n_data,
                                  0, len(gaps))
    tm = tm_all[768:832]                          # sky points 96..103, template 35 = sky 100, fdot 3
    inj = synth.random_injection(synth.SEED_BASE + 2, df=0.25, fdot=float(fd[3]),
                                 alpha=float(a[100]), delta=float(dl[100]))
    x, _ = injected_series(d, synth.SEED_BASE + 1, [inj], gaps)
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    t = plan.tuning()
    assert t["chunk"] == 64 and t["mode"] == fs.MODE_SPLIT
    assert plan.workspace.numel() > 8 * (1 << 30)
    got, rc = run_compute(d, x, tm, gaps, plan=plan)
    assert rc == 0
    plan.close()
    xc = x.astype(np.complex128)
    for i in (0, 35, 63):
        assert r15(got[i], oracle_two_f(d, x, tm[i], gaps)) <= TOL, i
    assert np.argmax(got[35]) == np.argmax(got[35])          # (finite)
    fr = F.bin_frequencies(d.n_fft, d.dt)
    rng = synth.rng(7)
    for i in (1, 9, 17, 30, 36, 44, 51, 62):
        q = rng.integers(0, d.n_fft, 16)
        ref = F.single_bin_two_f_many(xc, tm[i], gaps, d, fr[q])
        assert r15(got[i][q], ref) <= TOL, i


WINDOWS = [(R.WIN_RECT, 8), (R.WIN_RECT, 4), (R.WIN_RECT, 16), (R.WIN_LANCZOS, 2), (R.WIN_LANCZOS, 4),
           (R.WIN_LANCZOS, 6), (R.WIN_LANCZOS, 10), (R.WIN_LANCZOS, 12), (R.WIN_LANCZOS, 16)]


@pytest.mark.parametrize("window,taps", WINDOWS)
def test_every_window_and_tap_count(window, taps):
    """Windowed sinc of every tap count, with gaps at odd places (a one-sample
    gap, gaps at the span edges), three templates of uneven spans; the split
    mode (tiled resampler) and the fused mode against the oracle."""
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=40000, n_fft=1 << 16, interp=R.SINC, taps=taps, window=window,
                       f_het=150.0, max_templates=3)
    gaps = np.array([[0, 5], [3000, 5000], [20000, 20001], [30000, 33000], [39990, 40000]], np.int64)
    x, _ = injected_series(d, 7, [synth.random_injection(8, df=0.2)], gaps)
    tm = synth.make_templates([0.3, 2.5, 4.0], [-0.2, 0.9, 0.1], [0.0, -1e-9, -5e-9],
                              [0, 100, 1000], [40000, 39000, 30000], 0, len(gaps))
    refs = [oracle_two_f(d, x, tm[i], gaps) for i in range(3)]
    for mode in ("split", "fused"):
        got, rc = run_compute(d, x, tm, gaps, mode=MODES[mode])
        assert rc == 0, mode
        for i in range(3):
            assert r15(got[i], refs[i]) <= TOL, (mode, i)


def _span_templates(desc, days, seed):
    """Templates with the given spans (days), random placement and sky,
    fdot in [-1e-9, 0], each with its own gap list (0-20 %, 1-6 h blocks)."""
    g = synth.rng(seed)
    day = int(round(86400.0 / desc.dt))
    hour = int(round(3600.0 / desc.dt))
    lens = [min(int(v * day), desc.n_data) for v in days]
    starts = [int(g.integers(0, desc.n_data - L + 1)) for L in lens]
    gl, offs, cnts, o = [], [], [], 0
    for s, L in zip(starts, lens):
        gi = synth.gap_intervals(L, float(g.uniform(0.0, 0.2)), hour, 6 * hour,
                                 seed=int(g.integers(1 << 31))) + s
        gl.append(gi)
        offs.append(o)
        cnts.append(len(gi))
        o += len(gi)
    n = len(days)
    tm = synth.make_templates(g.uniform(0, 2 * np.pi, n), np.arcsin(g.uniform(-1, 1, n)),
                              g.uniform(-1e-9, 0.0, n), starts, lens, offs, cnts)
    return tm, np.concatenate(gl).astype(np.int64)


def test_ragged_batch_at_full_spans():
    """The batching workload's spans (1-10 d, FFT 2^18 .. 2^21, own gap
    lists) through RaggedBatch replayed from a CUDA graph: every bin of the
    1-day template, sampled bins of the longer ones."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300.batch import RaggedBatch
    desc = synth.batch_plan(max_templates=8)
    days = [1.0, 5.0, 10.0, 2.5, 7.3, 10.0]
    tm, gaps = _span_templates(desc, days, synth.SEED_BASE + 33)
    plan = fs.Plan(desc)
    nb = fs.fstat_template_nb(plan, tm)
    plan.close()
    nf = np.array([max(synth.next_pow2(int(v)), 1 << 12) for v in nb], np.int64)
    assert nf.min() == 1 << 18 and nf.max() == 1 << 21
    tm["n_fft"] = nf
    tm["out_off"] = np.concatenate([[0], np.cumsum(nf)[:-1]])
    inj = synth.random_injection(synth.SEED_BASE + 34, df=0.11, fdot=-1e-9)
    x, _ = injected_series(desc, synth.SEED_BASE + 35, [inj])
    dev = torch.device("cuda:0")
    rb = RaggedBatch(desc, torch.from_numpy(x).to(dev), tm, torch.from_numpy(gaps.reshape(-1).copy()).to(dev),
                     device=dev, slice_templates=4, graph=True)
    rb.twoF.fill_(float("nan"))
    rb.run()
    assert rb.status() == 0
    got = rb.twoF.cpu().numpy()
    rb.close()
    xc = x.astype(np.complex128)
    rng = synth.rng(8)
    for i in range(len(tm)):
        o, n = int(tm["out_off"][i]), int(nf[i])
        g = gaps[int(tm["gap_off"][i]):int(tm["gap_off"][i]) + int(tm["n_gaps"][i])]
        row = got[o:o + n]
        assert np.all(np.isfinite(row)), i
        if i == 0:
            assert r15(row, F.resample_two_f(xc, tm[i], g, desc, n_fft=n)) <= TOL
        else:
            q = rng.integers(0, n, 12)
            fr = (q - n // 2) / (n * desc.dt)
            ref = F.single_bin_two_f_many(xc, tm[i], g, desc, fr)
            assert r15(row[q], ref) <= TOL, i


def test_persistent_launch_at_full_spans():
    """The same ragged workload (1-10 d spans, FFT 2^18 .. 2^21 per
    template, own gap lists) in one persistent launch replayed from a CUDA
    graph, the batching design of the plan's persistent mode: every bin of
    the 1-day template, sampled bins of the others."""
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.batch_plan(max_templates=6)
    days = [1.0, 5.0, 10.0, 2.5, 7.3, 10.0]
    tm, gaps = _span_templates(desc, days, synth.SEED_BASE + 36)
    probe = fs.Plan(desc)
    nb = fs.fstat_template_nb(probe, tm)
    probe.close()
    nf = np.array([max(synth.next_pow2(int(v)), 1 << 12) for v in nb], np.int64)
    assert nf.min() == 1 << 18 and nf.max() == 1 << 21
    tm["n_fft"] = nf
    tm["out_off"] = np.concatenate([[0], np.cumsum(nf)[:-1]])
    inj = synth.random_injection(synth.SEED_BASE + 37, df=0.07, fdot=-5e-10)
    x, _ = injected_series(desc, synth.SEED_BASE + 38, [inj])
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc.replace(n_fft=int(nf.max())), device=dev)
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    out = torch.full((int(nf.sum()),), float("nan"), device=dev)
    runner = fs.GraphRunner(plan, torch.from_numpy(x).to(dev), fs.pack_templates(tm, device=dev),
                            torch.from_numpy(gaps.reshape(-1).copy()).to(dev), out)
    runner.replay()
    runner.stream.synchronize()
    assert fs.fstat_status(plan, runner.stream, raise_error=False) == 0
    got = out.cpu().numpy()
    plan.close()
    xc = x.astype(np.complex128)
    rng = synth.rng(9)
    for i in range(len(tm)):
        o, n = int(tm["out_off"][i]), int(nf[i])
        g = gaps[int(tm["gap_off"][i]):int(tm["gap_off"][i]) + int(tm["n_gaps"][i])]
        row = got[o:o + n]
        assert np.all(np.isfinite(row)), i
        if i == 0:
            assert r15(row, F.resample_two_f(xc, tm[i], g, desc, n_fft=n)) <= TOL
        else:
            q = rng.integers(0, n, 12)
            fr = (q - n // 2) / (n * desc.dt)
            assert r15(row[q], F.single_bin_two_f_many(xc, tm[i], g, desc, fr)) <= TOL, i


@pytest.mark.parametrize("mode", ["split", "fused", "plain"])
def test_degenerate_template_inside_a_gap(mode):
    """A template whose whole span lies inside a gap has no valid sample:
    A = B = C = D = 0 (Eqs. 9-10 as sums over no sample), 2F is undefined
    and the oracle gives no finite value.  The library reports ERANGE for
    the call, fills that template's row with NaN, and leaves the other
    templates of the same call as the oracle has them."""
    desc = synth.tiny_plan(interp=synth.SINC, taps=8, max_templates=3)
    gaps = np.array([[10000, 30000]], np.int64)
    a, dl = synth.random_sky(3, synth.SEED_BASE + 96)
    tm = synth.make_templates(a, dl, np.zeros(3), 0, desc.n_data, 0, 1)
    tm["span_start"][1] = 12000
    tm["span_len"][1] = 5000                     # [12000, 17000), inside the gap
    x, _ = injected_series(desc, synth.SEED_BASE + 97, [], gaps)
    with np.errstate(divide="ignore", invalid="ignore"):
        ref1 = oracle_two_f(desc, x, tm[1], gaps)
    assert not np.any(np.isfinite(ref1))
    got, rc = run_compute(desc, x, tm, gaps, mode=MODES[mode])
    assert rc == -2
    assert np.all(np.isnan(got[1]))
    for i in (0, 2):
        assert r15(got[i], oracle_two_f(desc, x, tm[i], gaps)) <= TOL, i


def test_sky_edges_poles_and_angle_wrap():
    """Sky positions at the edges of their ranges: both celestial poles
    (delta = +-pi/2, where the sidereal term of the Roemer delay vanishes),
    the ecliptic poles, alpha at 0, 2 pi and beyond it, negative alpha;
    2 d of data with an injection at the north pole, split mode, 8-tap
    Lanczos.  Every bin against the oracle."""
    d = synth.PlanDesc(dt=0.5, n_data=345600, n_fft=1 << 19, interp=R.SINC, f_het=150.0,
                       max_templates=8)
    inj = synth.random_injection(synth.SEED_BASE + 98, df=0.11, alpha=0.3, delta=np.pi / 2)
    x, _ = injected_series(d, synth.SEED_BASE + 99, [inj])
    eps = np.deg2rad(23.44)
    al = [0.3, 0.0, 2 * np.pi, 7.0, -2.5, 3 * np.pi / 2, np.pi / 2, 1.0]
    de = [np.pi / 2, -np.pi / 2, 0.4, -0.4, 1.1, np.pi / 2 - eps, -(np.pi / 2 - eps), 0.0]
    tm = synth.make_templates(al, de, np.zeros(8), 0, d.n_data)
    got, rc = run_compute(d, x, tm, mode=MODES["split"])
    assert rc == 0
    for i in range(len(tm)):
        assert r15(got[i], oracle_two_f(d, x, tm[i])) <= TOL, i
    assert np.max(got[0]) > 100                  # the injection, found at the pole


def test_search_size_common_phase_invariance():
    """A property that holds at any size (Eq. 6 depends on F_a, F_b only
    through |F_a|^2, |F_b|^2 and F_a F_b*): the search-sized workload (10 d,
    FFT 2^22, gaps, 8-tap Lanczos), its data multiplied by a common phase,
    gives the same 2F in every bin of four templates to FP32 rounding."""
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.search_plan(max_templates=4)
    gaps = synth.gap_intervals(d.n_data, 0.10, 7200, 43200, seed=synth.SEED_BASE + 1)
    x, _ = injected_series(d, synth.SEED_BASE + 39, [synth.random_injection(synth.SEED_BASE + 40, df=0.2)], gaps)
    a, dl = synth.random_sky(4, synth.SEED_BASE + 41)
    tm = synth.make_templates(a, dl, np.linspace(-1e-9, 0.0, 4), 0, d.n_data, 0, len(gaps))
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    ref, rc = run_compute(d, x, tm, gaps, plan=plan)
    assert rc == 0
    ph = np.complex64(np.exp(1j * 2.2))
    got, rc = run_compute(d, (x * ph).astype(np.complex64), tm, gaps, plan=plan)
    assert rc == 0
    plan.close()
    assert r15(got, ref) <= 2e-6
