"""Full-size precision and differentiation workloads against the FP64 oracle.

* Precision stress: 30 d at dt = 0.25 s (10,368,000 samples), FFT 2^24,
  f_h = 1 kHz, fdot = -1e-8 Hz/s, 8-tap sinc: all-FP64, mixed and all-FP32
  evaluation compared bin by bin with the oracle (max and median relative
  error), plus the SNR recovered at an injected signal.
* Differentiation: 5 d at dt = 0.5 s, 10 % gaps, 512 candidates scattered
  around 20 injections; the adjoint gradient of a sample of candidates
  against the oracle's central differences, then 50 preconditioned ascent
  steps for all 512.
The measured numbers are appended as JSON lines to the file
named by the FSTAT_RESULTS environment variable, if set."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import resample as R

from _gpu import NOGAPS, injected_series, r15, run_compute

pytestmark = pytest.mark.gpu


def _record(name, **kw):
    path = os.environ.get("FSTAT_RESULTS")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, **kw}) + "\n")


def test_precision_stress_all_modes():
    d0 = synth.stress_plan(max_templates=1)
    inj = synth.random_injection(synth.SEED_BASE + 3, df=0.123, fdot=-1e-8)
    x, info = injected_series(d0, synth.SEED_BASE + 3, [inj])
    tm = synth.make_templates(inj.alpha, inj.delta, inj.fdot, 0, d0.n_data)
    ref = F.resample_two_f(x.astype(np.complex128), tm[0], NOGAPS, d0)
    q_inj = int(np.argmax(ref))
    errs = {}
    for name, prec in (("fp64", synth.PREC_FP64), ("mixed", synth.PREC_MIXED), ("fp32", synth.PREC_FP32)):
        got, rc = run_compute(d0.replace(precision=prec), x, tm)
        assert rc == 0
        rel = np.abs(got[0].astype(np.float64) - ref) / np.maximum(ref, 4.0)
        errs[name] = (float(np.max(rel)), float(np.median(rel)), float(got[0][q_inj] / info[0][1]))
    _record("precision_stress", rho2=info[0][1], oracle_peak=float(ref[q_inj]),
            **{k: {"max_rel": v[0], "median_rel": v[1], "peak_over_rho2": v[2]} for k, v in errs.items()})
    # FP64 evaluation: measured 4.2e-7 max and 2.6e-8 median (the median is
    # the rounding of the float32 output); mixed: the parity tolerance
    assert errs["fp64"][0] <= 1e-6
    assert errs["mixed"][0] <= 1e-4
    # all-FP32 time map: the phase f_h t_m ~ 5e5 cycles cannot be held in FP32
    assert errs["fp32"][0] > 1e-2


def test_differentiation_workload():
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300.autograd import BinSearch, FStatBin, theta_of
    d = synth.diff_plan(max_templates=512)
    gaps = synth.gap_intervals(d.n_data, 0.10, 7200, 21600, seed=synth.SEED_BASE + 4)
    g = synth.rng(synth.SEED_BASE + 4)
    injs = [synth.random_injection(synth.SEED_BASE + 40 + i, df=float(g.uniform(-0.4, 0.4)),
                                   fdot=float(g.uniform(-1e-9, 0.0))) for i in range(20)]
    x, info = injected_series(d, synth.SEED_BASE + 4, injs, gaps)
    T = d.n_data * d.dt
    # candidates: offsets of 0.1-0.5 of a metric scale in every coordinate;
    # the sky scale is about c / (2 pi f v_orb T) ~ 4e-5 rad for 5 d near 100 Hz
    scale = np.array([1e-4, 1e-4, 1.0 / T, 1.0 / T ** 2])
    rows = []
    for c in range(512):
        inj = injs[c % 20]
        off = g.uniform(0.1, 0.5, 4) * g.choice([-1.0, 1.0], 4) * scale
        rows.append((inj.alpha + off[0], inj.delta + off[1], inj.df + off[2], inj.fdot + off[3]))
    rows = np.array(rows)
    tm = synth.make_templates(rows[:, 0], np.clip(rows[:, 1], -1.5, 1.5), rows[:, 3], 0, d.n_data, 0, len(gaps))
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    search = BinSearch(plan, torch.from_numpy(x).to(dev), tm, torch.from_numpy(gaps.reshape(-1).copy()).to(dev))
    theta = torch.tensor(theta_of(tm, rows[:, 2]), device=dev)
    th = theta.clone().requires_grad_(True)
    y = FStatBin.apply(th, search)
    y.sum().backward()
    grad = th.grad.cpu().numpy()
    y = y.detach()
    assert fs.fstat_status(plan, raise_error=False) == 0
    xc = x.astype(np.complex128)
    worst = 0.0
    for i in (0, 137, 301):
        ref = F.single_bin_gradient(xc, tm[i], gaps, d, rows[i, 2])
        ref2f = F.single_bin_two_f(xc, tm[i], gaps, d, rows[i, 2])
        assert abs(float(y[i]) - ref2f) / max(ref2f, 4.0) < 1e-4
        err = np.linalg.norm((grad[i] - ref) * scale) / max(np.linalg.norm(ref * scale), 1e-3 * ref2f)
        worst = max(worst, err)
    # 50 steps of normalised, preconditioned gradient ascent
    truth = np.array([[j.alpha, j.delta, j.df, j.fdot] for j in injs])
    true_tm = synth.make_templates(truth[:, 0], truth[:, 1], truth[:, 3], 0, d.n_data, 0, len(gaps))
    tsearch = BinSearch(plan, search.x_h, true_tm, search.gaps)
    true2f = FStatBin.apply(torch.tensor(truth, device=dev), tsearch).detach().cpu().numpy()
    sc = torch.tensor(scale, device=dev)
    start = y.detach().cpu().numpy()
    for it in range(50):
        th = theta.clone().requires_grad_(True)
        FStatBin.apply(th, search).sum().backward()
        gr = th.grad * sc
        norm = torch.sqrt((gr ** 2).sum(1, keepdim=True)).clamp_min(1e-30)
        theta = theta + gr * sc / norm * (0.5 * 0.9 ** it + 0.01)
    final = FStatBin.apply(theta, search).detach().cpu().numpy()
    frac = final / true2f[np.arange(512) % 20]
    _record("differentiation", fd_worst_rel=worst, start_median_frac=float(np.median(start / true2f[np.arange(512) % 20])),
            final_median_frac=float(np.median(frac)), final_p10_frac=float(np.percentile(frac, 10)))
    assert worst < 1e-3
    assert np.median(frac) > 0.9
