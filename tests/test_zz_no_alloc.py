"""The allocation-free entry point against fstat_compute.

fstat_compute_noalloc serves callers that cannot allocate device memory (a
plugin inside a framework that owns the memory pool, a real-time loop that
cannot take cudaMalloc's synchronisation): it uses a fixed scratch array
inside the library instead of a plan and a caller workspace.  Two calls in a
row, with different templates, must each give what fstat_compute gives on
the same inputs, within the parity tolerance of the other GPU tests.  This
file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

import synth
from oracle import resample as R

from _gpu import injected_series, r15, run_compute

pytestmark = pytest.mark.gpu
TOL = 1e-4


def test_noalloc_matches_compute_on_two_calls():
    import torch
    import paper_0912_4255_gb300 as fs
    d = synth.PlanDesc(dt=0.5, n_data=120_000, n_fft=1 << 17, interp=R.SINC, f_het=120.0,
                       max_templates=3)
    gaps = synth.gap_intervals(d.n_data, 0.1, 3600, 9000, seed=12)
    x, _ = injected_series(d, 13, [synth.random_injection(14, df=0.3)], gaps)
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(x).to(dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    batches = [
        synth.make_templates([0.4, 2.0, 5.0], [0.1, -0.7, 1.2], [0.0, -1e-9, -4e-9],
                             [0, 1000, 0], [120_000, 100_000, 90_000], 0, len(gaps)),
        synth.make_templates([1.5, 3.3], [-1.1, 0.6], [-2e-9, 0.0], [500, 0],
                             [110_000, 120_000], 0, len(gaps)),
    ]
    for tm in batches:
        ref, rc = run_compute(d, x, tm, gaps)
        assert rc == 0
        out = fs.fstat_compute_noalloc(d, xd, fs.pack_templates(tm, device=dev), gd)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(tm), -1)
        assert np.all(np.isfinite(got))
        for i in range(len(tm)):
            assert r15(got[i], ref[i]) <= TOL, i


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
