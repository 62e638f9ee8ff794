"""The allocation-free entry point against fstat_compute and the oracle.

fstat_compute_noalloc serves callers that cannot allocate device memory (a
plugin inside a framework that owns the memory pool, a real-time loop that
cannot take cudaMalloc's synchronisation): it uses a fixed scratch array
inside the library instead of a plan and a caller workspace.  Two calls in a
row, with different templates, must each give what fstat_compute gives on
the same inputs, within the parity tolerance of the other GPU tests, and
match the FP64 oracle to the same tolerance; the first call of a process,
made before any plan exists, must do so as well.  This file is collected
last so that a failure here leaves every other test run.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import resample as R

from _gpu import injected_series, oracle_two_f, r15, run_compute

pytestmark = pytest.mark.gpu
TOL = 1e-4
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "sinc8": dict(interp=R.SINC, taps=8),
    "nearest": dict(interp=R.NEAREST),
    "sinc4": dict(interp=R.SINC, taps=4),
    "sinc16": dict(interp=R.SINC, taps=16),
    "rect6": dict(interp=R.SINC, taps=6, window=R.WIN_RECT),
    "fp32": dict(interp=R.SINC, taps=8, precision=synth.PREC_FP32),
}


def _inputs(**kw):
    d = synth.PlanDesc(dt=0.5, n_data=120_000, n_fft=1 << 17, f_het=120.0, max_templates=3, **kw)
    gaps = synth.gap_intervals(d.n_data, 0.1, 3600, 9000, seed=12)
    x, _ = injected_series(d, 13, [synth.random_injection(14, df=0.3)], gaps)
    batches = [
        synth.make_templates([0.4, 2.0, 5.0], [0.1, -0.7, 1.2], [0.0, -1e-9, -4e-9],
                             [0, 1000, 0], [120_000, 100_000, 90_000], 0, len(gaps)),
        synth.make_templates([1.5, 3.3], [-1.1, 0.6], [-2e-9, 0.0], [500, 0],
                             [110_000, 120_000], 0, len(gaps)),
    ]
    return d, gaps, x, batches


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_compute_on_two_calls(case):
    import torch
    import paper_0912_4255_gb300 as fs
    d, gaps, x, batches = _inputs(**CASES[case])
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(x).to(dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    for tm in batches:
        ref, rc = run_compute(d, x, tm, gaps)
        assert rc == 0
        out = torch.full((len(tm) * d.n_fft,), float("nan"), device=dev)
        fs.fstat_compute_noalloc(d, xd, fs.pack_templates(tm, device=dev), gd, twoF=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(tm), -1)
        assert np.all(np.isfinite(got))
        for i in range(len(tm)):
            assert r15(got[i], ref[i]) <= TOL, (case, i)


@pytest.mark.parametrize("case", ["sinc8", "nearest", "sinc16"])
def test_noalloc_matches_the_oracle(case):
    """Directly against the FP64 oracle of the same algorithm (mixed
    precision; the FP32 mode cannot hold the heterodyne phase)."""
    import torch
    import paper_0912_4255_gb300 as fs
    d, gaps, x, batches = _inputs(**CASES[case])
    dev = torch.device("cuda:0")
    tm = batches[0]
    out = fs.fstat_compute_noalloc(d, torch.from_numpy(x).to(dev), fs.pack_templates(tm, device=dev),
                                   torch.from_numpy(gaps.reshape(-1).copy()).to(dev))
    got = out.cpu().numpy().reshape(len(tm), -1)
    for i in (0, 2):
        assert r15(got[i], oracle_two_f(d, x, tm[i], gaps)) <= TOL, (case, i)


_FRESH = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import paper_0912_4255_gb300 as fs
from test_zz_no_alloc import _inputs
d, gaps, x, batches = _inputs(interp=1, taps=8)
dev = torch.device("cuda:0")
xd = torch.from_numpy(x).to(dev)
gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
outs = []
for tm in batches:        # two calls, the first one before any plan exists
    out = torch.empty(len(tm) * d.n_fft, device=dev)
    fs.fstat_compute_noalloc(d, xd, fs.pack_templates(tm, device=dev), gd, twoF=out)
    torch.cuda.synchronize()
    outs.append(out.cpu().numpy())
np.save(sys.argv[2], np.concatenate(outs))
"""


def test_noalloc_first_call_in_a_fresh_process(tmp_path):
    """The first call of a process does the set-up (the array's device
    address, the tables): run it in a new interpreter before any plan is
    created there, then compare both calls with fstat_compute here."""
    dst = str(tmp_path / "fresh.npy")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT, dst], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(dst)
    d, gaps, x, batches = _inputs(interp=R.SINC, taps=8)
    o = 0
    for tm in batches:
        ref, rc = run_compute(d, x, tm, gaps)
        assert rc == 0
        g = got[o:o + len(tm) * d.n_fft].reshape(len(tm), -1)
        o += len(tm) * d.n_fft
        for i in range(len(tm)):
            assert r15(g[i], ref[i]) <= TOL, i


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=1000, n_fft=1 << 21, interp=R.NEAREST, max_templates=1)
    dev = torch.device("cuda:0")
    x = torch.zeros(d.n_data, dtype=torch.complex64, device=dev)
    tm = fs.pack_templates(synth.make_templates(1.0, 0.0, 0.0, 0, d.n_data), device=dev)
    with pytest.raises(fs.FstatError) as e:
        fs.fstat_compute_noalloc(d, x, tm, twoF=torch.empty(1 << 21, device=dev))
    assert e.value.code == fs._lib.FSTAT_ERANGE
    # FP64 is not offered; a short output buffer is refused before the call
    with pytest.raises(fs.FstatError) as e:
        fs.fstat_compute_noalloc(d.replace(n_fft=1 << 14, precision=synth.PREC_FP64), x, tm)
    assert e.value.code == fs._lib.FSTAT_ENOTSUP
    with pytest.raises(ValueError):
        fs.fstat_compute_noalloc(d.replace(n_fft=1 << 14), x, tm, twoF=torch.empty(100, device=dev))


def test_noalloc_refuses_host_memory():
    """Pointers the current GPU cannot use are refused on the host, before
    any launch (a host buffer passed as twoF)."""
    import ctypes
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import _lib
    d = synth.PlanDesc(dt=0.5, n_data=1000, n_fft=1 << 14, interp=R.NEAREST, max_templates=1)
    dev = torch.device("cuda:0")
    x = torch.zeros(d.n_data, dtype=torch.complex64, device=dev)
    tm = fs.pack_templates(synth.make_templates(1.0, 0.0, 0.0, 0, d.n_data), device=dev)
    host = torch.empty(1 << 14, dtype=torch.float32)
    rc = _lib.load().fstat_compute_noalloc(ctypes.byref(fs._desc(d)), ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(tm.data_ptr()), 1, ctypes.c_void_p(0), 0,
                                           ctypes.c_void_p(host.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.FSTAT_EINVAL


def test_noalloc_at_its_largest_fft():
    """n_fft = 2^20, the largest length the fixed scratch array holds (3.6 d
    at 0.5 s, two templates, gaps): against fstat_compute and, for every bin
    of the first template, against the oracle."""
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=620_000, n_fft=1 << 20, f_het=120.0, max_templates=2,
                       interp=R.SINC, taps=8)
    gaps = synth.gap_intervals(d.n_data, 0.1, 3600, 21600, seed=15)
    x, _ = injected_series(d, 16, [synth.random_injection(17, df=0.2)], gaps)
    tm = synth.make_templates([0.7, 4.1], [0.2, -0.9], [0.0, -2e-9], [0, 3000], [620_000, 600_000],
                              0, len(gaps))
    ref, rc = run_compute(d, x, tm, gaps)
    assert rc == 0
    dev = torch.device("cuda:0")
    out = torch.full((2 * d.n_fft,), float("nan"), device=dev)
    fs.fstat_compute_noalloc(d, torch.from_numpy(x).to(dev), fs.pack_templates(tm, device=dev),
                             torch.from_numpy(gaps.reshape(-1).copy()).to(dev), twoF=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(2, -1)
    for i in range(2):
        assert r15(got[i], ref[i]) <= TOL, i
    assert r15(got[0], oracle_two_f(d, x, tm[0], gaps)) <= TOL
