"""The autotuner on a small plan: it times the candidates, keeps the ones
that reproduce the default tuning, sets the fastest, and the plan then
still matches the oracle."""
import numpy as np
import pytest

import synth
from oracle import resample as R

from _gpu import injected_series, oracle_two_f, r15

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_valid_shape(tmp_path):
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import autotune as at
    d = synth.PlanDesc(dt=0.5, n_data=100_000, n_fft=1 << 17, interp=R.SINC, f_het=60.0,
                       max_templates=8)
    gaps = synth.gap_intervals(d.n_data, 0.1, 3600, 9000, seed=21)
    x, _ = injected_series(d, 22, [synth.random_injection(23, df=0.15)], gaps)
    a, de = synth.fibonacci_sky(8)
    tm = synth.make_templates(a, de, np.linspace(-1e-9, 0, 8), 0, d.n_data, 0, len(gaps))
    dev = torch.device("cuda:0")
    plan = fs.Plan(d, device=dev)
    xd = torch.from_numpy(x).to(dev)
    td = fs.pack_templates(tm, device=dev)
    gd = torch.from_numpy(gaps.reshape(-1).copy()).to(dev)
    cache = str(tmp_path / "tune.json")
    res = at.autotune(plan, xd, td, gd, repeats=2, cache=cache)
    assert not res["cached"]
    timed = [r for r in res["results"] if "skipped" not in r]
    assert len(timed) >= 5
    assert all(r["err"] is None or r["err"] < 1e-4 for r in timed)
    assert plan.tuning()["mode"] == res["tuning"]["mode"]
    got = fs.fstat_compute(plan, xd, td, gd).cpu().numpy().reshape(8, -1)
    assert fs.fstat_status(plan, raise_error=False) == 0
    for i in (0, 5):
        assert r15(got[i], oracle_two_f(d, x, tm[i], gaps)) <= 1e-4
    # a second plan of the same shape takes the cached choice
    plan2 = fs.Plan(d, device=dev)
    assert at.apply_cached(plan2, cache)
    assert plan2.tuning()["mode"] == res["tuning"]["mode"]
    again = at.autotune(plan2, xd, td, gd, cache=cache)
    assert again["cached"]


def test_default_knot_spacing_matches_the_host_rule():
    """The plan's default knot spacing is the rule the autotuner mirrors:
    2^11 points for the searches at 0.5 s and 100 Hz, 2^10 up to 100 cycles
    per sample, 2^9 beyond, and 2^10 at dt = 1 s."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import autotune as at
    for f_het, dt, want in [(100.0, 0.5, 11), (150.0, 0.5, 10), (1000.0, 0.25, 9), (40.0, 1.0, 10)]:
        d = synth.PlanDesc(dt=dt, n_data=50000, n_fft=1 << 17, f_het=f_het, max_templates=1)
        plan = fs.Plan(d, device=torch.device("cuda:0"))
        assert plan.tuning()["knot_log2"] == want == at.default_knot_log2(f_het, dt)
        plan.close()
