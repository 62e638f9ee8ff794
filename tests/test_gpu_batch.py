"""Batched execution: one persistent launch over templates with uneven
spans, per-template gap lists and per-template FFT lengths (next power of two
of the resampled length), under a CUDA graph; against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import resample as R

from _gpu import MODES, injected_series, r15, run_compute

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _ragged_batch(n, seed, desc, min_days=0.15, max_days=0.45):
    tm, gaps = synth.batch_templates(n, desc.n_data, desc.dt, seed, min_days=min_days,
                                     max_days=max_days, max_gap_frac=0.2)
    import paper_0912_4255_gb300 as fs
    plan = fs.Plan(desc)
    nb = fs.fstat_template_nb(plan, tm)
    plan.close()
    nf = np.array([max(synth.next_pow2(int(v)), 1 << 12) for v in nb], np.int64)
    tm["n_fft"] = nf
    tm["out_off"] = np.concatenate([[0], np.cumsum(nf)[:-1]])
    return tm, gaps, nf


def _data(desc, seed, gaps_all):
    # shared series: noise (gaps are per template masks, the data itself has none)
    inj = synth.random_injection(seed, df=0.11, fdot=-1e-9)
    x, _ = injected_series(desc, seed, [inj])
    return x


def test_persistent_ragged_batch_matches_oracle():
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.PlanDesc(dt=0.5, n_data=86400, n_fft=1 << 17, interp=R.SINC, f_het=100.0,
                          max_templates=10)
    tm, gaps, nf = _ragged_batch(10, 61, desc)
    assert len(set(nf.tolist())) >= 2          # really ragged
    x = _data(desc, 62, gaps)
    plan = fs.Plan(desc)
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    dev = torch.device("cuda:0")
    out = torch.full((int(nf.sum()),), float("nan"), dtype=torch.float32, device=dev)
    fs.fstat_compute(plan, torch.from_numpy(x).to(dev), fs.pack_templates(tm, device=dev),
                     torch.from_numpy(gaps.reshape(-1).copy()).to(dev), out)
    assert fs.fstat_status(plan, raise_error=False) == 0
    got = out.cpu().numpy()
    for i in range(len(tm)):
        o, n = int(tm["out_off"][i]), int(nf[i])
        g = gaps[int(tm["gap_off"][i]):int(tm["gap_off"][i]) + int(tm["n_gaps"][i])]
        ref = F.resample_two_f(x.astype(np.complex128), tm[i], g, desc, n_fft=n)
        assert r15(got[o:o + n], ref) <= TOL, i


def test_ragged_batch_in_split_groups():
    """The same kind of ragged batch through RaggedBatch (one split-mode plan
    per FFT length, every 2F at its template's out_off, replayed from a CUDA
    graph) against the oracle, and against the persistent launch."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300.batch import RaggedBatch
    desc = synth.PlanDesc(dt=0.5, n_data=86400, n_fft=1 << 17, interp=R.SINC, f_het=100.0,
                          max_templates=12)
    tm, gaps, nf = _ragged_batch(12, 63, desc)
    assert len(set(nf.tolist())) >= 2
    x = _data(desc, 64, gaps)
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(x).to(dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    rb = RaggedBatch(desc, xd, tm, gd, device=dev, slice_templates=4, graph=True)
    rb.twoF.fill_(float("nan"))
    torch.cuda.synchronize()
    rb.run()
    assert rb.status() == 0                   # synchronises the batch's stream
    got = rb.twoF.cpu().numpy()
    for i in range(len(tm)):
        o, n = int(tm["out_off"][i]), int(nf[i])
        g = gaps[int(tm["gap_off"][i]):int(tm["gap_off"][i]) + int(tm["n_gaps"][i])]
        ref = F.resample_two_f(x.astype(np.complex128), tm[i], g, desc, n_fft=n)
        assert r15(got[o:o + n], ref) <= TOL, i
    plan = fs.Plan(desc)
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    per = torch.empty_like(rb.twoF)
    fs.fstat_compute(plan, xd, fs.pack_templates(tm, device=dev), gd, per)
    assert fs.fstat_status(plan, raise_error=False) == 0
    assert r15(got, per.cpu().numpy()) < 1e-5
    rb.close()


def test_persistent_equals_fused_and_graph_replay():
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.PlanDesc(dt=0.5, n_data=100_000, n_fft=1 << 17, interp=R.SINC, f_het=90.0,
                          max_templates=7)
    gaps = synth.gap_intervals(desc.n_data, 0.1, 3600, 9000, seed=5)
    x, _ = injected_series(desc, 71, [synth.random_injection(72, df=0.2)], gaps)
    a, d = synth.fibonacci_sky(7)
    tm = synth.make_templates(a, d, np.linspace(-2e-9, 0, 7), 0, desc.n_data, 0, len(gaps))
    ref, rc = run_compute(desc, x, tm, gaps, mode=MODES["fused"])
    assert rc == 0
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc)
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    xd = torch.from_numpy(x).to(dev)
    td = fs.pack_templates(tm, device=dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    eager = fs.fstat_compute(plan, xd, td, gd).cpu().numpy().reshape(len(tm), -1)
    assert fs.fstat_status(plan, raise_error=False) == 0
    # the two modes sum A, B, C over first-pass tiles of different sizes
    # (8k points per persistent work item, 16k per fused block): they agree
    # to the rounding of those sums
    assert r15(eager, ref) < 1e-5
    runner = fs.GraphRunner(plan, xd, td, gd)
    runner.twoF.fill_(0)
    for _ in range(2):
        got = runner.replay()
    torch.cuda.synchronize()
    assert fs.fstat_status(plan, raise_error=False) == 0
    assert np.array_equal(got.cpu().numpy().reshape(len(tm), -1), eager)


def test_split_graph_replay_matches_eager():
    """The default (split) mode captured in a CUDA graph: the resampler, the
    A/B/C reduction and both passes replay bit for bit, and agree with the
    fused mode to rounding of the sums."""
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.PlanDesc(dt=0.5, n_data=100_000, n_fft=1 << 17, interp=R.SINC, f_het=90.0,
                          max_templates=7)
    gaps = synth.gap_intervals(desc.n_data, 0.1, 3600, 9000, seed=6)
    x, _ = injected_series(desc, 73, [synth.random_injection(74, df=-0.2)], gaps)
    a, d = synth.fibonacci_sky(7)
    tm = synth.make_templates(a, d, np.linspace(-2e-9, 0, 7), 0, desc.n_data, 0, len(gaps))
    fused, rc = run_compute(desc, x, tm, gaps, mode=MODES["fused"])
    assert rc == 0
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc)
    assert plan.tuning()["mode"] == fs.MODE_SPLIT
    xd = torch.from_numpy(x).to(dev)
    td = fs.pack_templates(tm, device=dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    eager = fs.fstat_compute(plan, xd, td, gd).cpu().numpy().reshape(len(tm), -1)
    assert fs.fstat_status(plan, raise_error=False) == 0
    assert r15(eager, fused) < 1e-5
    runner = fs.GraphRunner(plan, xd, td, gd)
    runner.twoF.fill_(0)
    for _ in range(2):
        got = runner.replay()
    torch.cuda.synchronize()
    assert fs.fstat_status(plan, raise_error=False) == 0
    assert np.array_equal(got.cpu().numpy().reshape(len(tm), -1), eager)


def test_persistent_bounded_wait_reports_timeout_and_recovers():
    """A row block made to wait for a column tile that never runs gives up
    after its iteration limit: the call reports FSTAT_ETIMEOUT and the plan
    keeps working."""
    import torch
    import paper_0912_4255_gb300 as fs
    desc = synth.PlanDesc(dt=0.5, n_data=30_000, n_fft=1 << 15, interp=R.NEAREST, max_templates=4)
    x = synth.complex_noise(desc.n_data, 1.0, 3)
    tm = synth.make_templates([0.1, 1.1, 2.1, 3.1], 0.3, 0.0, 0, desc.n_data)
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc)
    plan.set_tuning(mode=fs.MODE_PERSISTENT)
    xd = torch.from_numpy(x).to(dev)
    td = fs.pack_templates(tm, device=dev)
    fs.fstat_debug_stall(plan, 1)
    fs.fstat_compute(plan, xd, td)
    assert fs.fstat_status(plan, raise_error=False) == fs._lib.FSTAT_ETIMEOUT
    good = fs.fstat_compute(plan, xd, td).cpu().numpy().reshape(4, -1)
    assert fs.fstat_status(plan, raise_error=False) == 0
    # a fresh plan in the same mode gives the same bits
    ref, rc = run_compute(desc, x, tm, mode=MODES["persistent"])
    assert rc == 0 and np.array_equal(good, ref)
