"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on
seeded inputs and compare with the FP64 oracle."""
import numpy as np

import synth
from oracle import fstat as F
from oracle import inject as I
from oracle import resample as R

NOGAPS = np.zeros((0, 2), np.int64)
# FSTAT_MODE_* of include/fstat.h
MODES = {"fused": 0, "plain": 1, "persistent": 2, "split": 3}


def r15(got, ref):
    """max_q |2F_gpu - 2F_oracle| / max(2F_oracle, 4): relative error with a
    floor at the noise mean, so that bins near zero do not dominate."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(ref, 4.0)))


def device():
    import torch
    return torch.device("cuda:0")


def run_compute(desc, x, templates, gaps=NOGAPS, mode=None, tuning=None, plan=None):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = device()
    own = plan is None
    if own:
        plan = fs.Plan(desc, device=dev)
    if mode is not None or tuning:
        plan.set_tuning(mode=fs.MODE_SPLIT if mode is None else mode, **(tuning or {}))
    xd = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).to(dev)
    td = fs.pack_templates(templates, device=dev)
    gd = torch.from_numpy(np.ascontiguousarray(gaps, np.int64).reshape(-1)).to(dev)
    out = fs.fstat_compute(plan, xd, td, gd)
    rc = fs.fstat_status(plan, raise_error=False)
    res = out.cpu().numpy().reshape(len(templates), -1)
    if own:
        plan.close()
    return res, rc


def run_resample(desc, x, templates, gaps=NOGAPS):
    import torch
    import paper_0912_4255_gb300 as fs
    dev = device()
    plan = fs.Plan(desc, device=dev)
    xd = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).to(dev)
    td = fs.pack_templates(templates, device=dev)
    gd = torch.from_numpy(np.ascontiguousarray(gaps, np.int64).reshape(-1)).to(dev)
    wa, wb, abcd = fs.fstat_resample(plan, xd, td, gd)
    rc = fs.fstat_status(plan, raise_error=False)
    out = wa.cpu().numpy(), wb.cpu().numpy(), abcd.cpu().numpy()
    plan.close()
    return out, rc


def oracle_two_f(desc, x, tmpl, gaps=NOGAPS):
    return F.resample_two_f(np.asarray(x, np.complex64).astype(np.complex128), tmpl,
                            _template_gaps(tmpl, gaps), desc)


def _template_gaps(tmpl, gaps):
    o, n = int(tmpl["gap_off"]), int(tmpl["n_gaps"])
    return np.asarray(gaps, np.int64).reshape(-1, 2)[o:o + n]


def tie_margin(desc, tmpl):
    """Distance of the NN decisions from a rounding tie (FP64)."""
    from oracle import timemap as TM
    _, T, _ = TM.resample_times(tmpl, desc)
    return R.nn_tie_margin(R.fractional_index(T, desc))


def injected_series(desc, seed, injections, gaps=NOGAPS):
    noise = synth.complex_noise(desc.n_data, desc.sigma2, seed)
    valid = I.valid_all(desc, gaps)
    noise = np.where(valid, noise, 0)
    x, info = I.inject(noise, injections, desc, valid)
    return x.astype(np.complex64), info
