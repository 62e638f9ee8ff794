"""Gradient of 2F at a chosen bin: the adjoint kernel against the FP64 oracle's
central-difference gradient, the autograd wrapper, and gradient ascent
towards injected signals."""
import numpy as np
import pytest

import synth
from oracle import fstat as F
from oracle import resample as R

from _gpu import injected_series

pytestmark = pytest.mark.gpu


def _grad_gpu(desc, x, tm, df, gaps):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = torch.device("cuda:0")
    plan = fs.Plan(desc, device=dev)
    xd = torch.from_numpy(x).to(dev)
    td = fs.pack_templates(tm, device=dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    two_f, grad = fs.fstat_grad(plan, xd, td, torch.as_tensor(df, dtype=torch.float64), gd)
    rc = fs.fstat_status(plan, raise_error=False)
    out = two_f.cpu().numpy(), grad.cpu().numpy()
    plan.close()
    return out, rc


def _setup(n_data, seed, n_inj=2, gap_frac=0.1):
    d = synth.PlanDesc(dt=0.5, n_data=n_data, n_fft=synth.next_pow2(n_data + 64), interp=R.SINC,
                       f_het=100.0, max_templates=16)
    gaps = synth.gap_intervals(n_data, gap_frac, 3600, 12000, seed=seed)
    injs = [synth.random_injection(seed + i, df=0.05 + 0.1 * i, fdot=-1e-9 * (i + 1)) for i in range(n_inj)]
    x, info = injected_series(d, seed, injs, gaps)
    return d, gaps, injs, x


def test_adjoint_matches_fp64_central_differences():
    """Candidates offset from two injections (within a fraction of the
    metric scale) plus noise-only points; 2F within 1e-4 and the gradient
    within 1e-3 (scaled by the metric scales) of the oracle's central
    differences with Richardson extrapolation."""
    d, gaps, injs, x = _setup(100_000, 50)
    T = d.n_data * d.dt
    g = synth.rng(3)
    al, de, fd, df = [], [], [], []
    for inj in injs:
        for _ in range(2):
            al.append(inj.alpha + g.uniform(-2e-3, 2e-3))
            de.append(inj.delta + g.uniform(-2e-3, 2e-3))
            fd.append(inj.fdot + g.uniform(-0.3, 0.3) / T ** 2)
            df.append(inj.df + g.uniform(-0.3, 0.3) / T)
    al.append(1.0); de.append(0.2); fd.append(0.0); df.append(0.11)
    tm = synth.make_templates(al, de, fd, 0, d.n_data, 0, len(gaps))
    (two_f, grad), rc = _grad_gpu(d, x, tm, np.array(df), gaps)
    assert rc == 0
    xc = x.astype(np.complex128)
    scale = np.array([1e-3, 1e-3, 1.0 / T, 1.0 / T ** 2])
    for i in range(len(tm)):
        ref2f = F.single_bin_two_f(xc, tm[i], gaps, d, df[i])
        assert abs(two_f[i] - ref2f) / max(ref2f, 4.0) < 1e-4
        ref = F.single_bin_gradient(xc, tm[i], gaps, d, df[i])
        err = np.linalg.norm((grad[i] - ref) * scale) / max(np.linalg.norm(ref * scale), 1e-3 * max(ref2f, 4.0))
        assert err < 1e-3, (i, grad[i], ref)


def test_adjoint_with_second_spindown():
    """The adjoint's phase rate includes the second spindown: gradient
    against the oracle's central differences for templates with fddot."""
    d, gaps, injs, x = _setup(100_000, 57, n_inj=1)
    T = d.n_data * d.dt
    inj = injs[0]
    tm = synth.make_templates([inj.alpha, inj.alpha + 1e-3], [inj.delta, inj.delta - 1e-3],
                              [inj.fdot, inj.fdot + 0.2 / T ** 2], 0, d.n_data, 0, len(gaps),
                              fddot=[2e-14, -3e-14])
    df = np.array([inj.df, inj.df + 0.1 / T])
    (two_f, grad), rc = _grad_gpu(d, x, tm, df, gaps)
    assert rc == 0
    xc = x.astype(np.complex128)
    scale = np.array([1e-3, 1e-3, 1.0 / T, 1.0 / T ** 2])
    for i in range(2):
        ref2f = F.single_bin_two_f(xc, tm[i], gaps, d, df[i])
        assert abs(two_f[i] - ref2f) / max(ref2f, 4.0) < 1e-4
        ref = F.single_bin_gradient(xc, tm[i], gaps, d, df[i])
        err = np.linalg.norm((grad[i] - ref) * scale) / max(np.linalg.norm(ref * scale), 1e-3 * max(ref2f, 4.0))
        assert err < 1e-3, (i, grad[i], ref)


def test_autograd_function_backward():
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300.autograd import BinSearch, FStatBin, theta_of
    d, gaps, injs, x = _setup(60_000, 70, n_inj=1)
    tm = synth.make_templates([injs[0].alpha + 1e-3, 2.0], [injs[0].delta, -0.5],
                              [injs[0].fdot, 0.0], 0, d.n_data, 0, len(gaps))
    df = [injs[0].df + 2e-6, 0.3]
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    search = BinSearch(plan, torch.from_numpy(x).to(dev), tm,
                       torch.from_numpy(gaps.reshape(-1).copy()).to(dev))
    theta = torch.tensor(theta_of(tm, df), device=dev, requires_grad=True)
    y = FStatBin.apply(theta, search)
    (y * torch.tensor([1.0, 2.0], device=dev, dtype=torch.float64)).sum().backward()
    (two_f, grad), _ = _grad_gpu(d, x, tm, np.array(df), gaps)
    np.testing.assert_allclose(y.detach().cpu().numpy(), two_f, rtol=1e-12)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), grad * np.array([[1.0], [2.0]]), rtol=1e-12)


def test_gradient_ascent_recovers_injections():
    """50 preconditioned gradient-ascent steps from offset candidates recover
    most of the true 2F of each injection."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300.autograd import BinSearch, FStatBin, theta_of
    d, gaps, injs, x = _setup(200_000, 90, n_inj=3)
    T = d.n_data * d.dt
    g = synth.rng(9)
    tm = synth.make_templates([i.alpha + g.uniform(-1e-3, 1e-3) for i in injs],
                              [i.delta + g.uniform(-1e-3, 1e-3) for i in injs],
                              [i.fdot for i in injs], 0, d.n_data, 0, len(gaps))
    df0 = np.array([i.df + g.uniform(-0.4, 0.4) / T for i in injs])
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    search = BinSearch(plan, torch.from_numpy(x).to(dev), tm,
                       torch.from_numpy(gaps.reshape(-1).copy()).to(dev))
    truth = synth.make_templates([i.alpha for i in injs], [i.delta for i in injs],
                                 [i.fdot for i in injs], 0, d.n_data, 0, len(gaps))
    true_2f = FStatBin.apply(torch.tensor(theta_of(truth, [i.df for i in injs]), device=dev),
                             search).detach()
    theta = torch.tensor(theta_of(tm, df0), device=dev)
    scale = torch.tensor([2e-3, 2e-3, 0.5 / T, 0.5 / T ** 2], device=dev, dtype=torch.float64)
    start = None
    for it in range(50):
        th = theta.clone().requires_grad_(True)
        y = FStatBin.apply(th, search)
        if start is None:
            start = y.detach()
        y.sum().backward()
        step = th.grad * scale * scale
        norm = torch.sqrt(((th.grad * scale) ** 2).sum(1, keepdim=True)).clamp_min(1e-30)
        theta = theta + step / norm * (0.5 * 0.9 ** it + 0.01)
    final = FStatBin.apply(theta, search).detach()
    frac = (final / true_2f).cpu().numpy()
    assert np.all(frac > 0.9), (frac, (start / true_2f).cpu().numpy())
