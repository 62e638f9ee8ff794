"""Host logic of the autotuner: candidate shapes, selection under the
accuracy guard, and the cache (no GPU)."""
import synth
from paper_0912_4255_gb300 import autotune as at
from paper_0912_4255_gb300._lib import MODE_FUSED, MODE_PERSISTENT, MODE_SPLIT


def test_candidates_cover_every_valid_factorisation():
    d = synth.search_plan(max_templates=64)                 # 2^22
    c = at.candidates(d)
    assert c[0] == {"mode": MODE_SPLIT}                     # the reference comes first
    split_l1 = sorted(t["log2_n1"] for t in c if t.get("mode") == MODE_SPLIT and "log2_n1" in t)
    assert split_l1 == [10, 11, 12]                         # N1, N2 within 2^6 .. 2^12
    assert {t["mode"] for t in c} == {MODE_SPLIT, MODE_FUSED, MODE_PERSISTENT}
    assert {"mode": MODE_SPLIT, "knot_log2": 10} in c       # denser knots only (the default is 11 here)
    small = synth.PlanDesc(dt=0.5, n_data=60000, n_fft=1 << 17, max_templates=4)
    assert sorted(t["log2_n1"] for t in at.candidates(small) if t.get("mode") == MODE_SPLIT
                  and "log2_n1" in t) == [6, 7, 8, 9, 10, 11]


def test_cache_key_depends_on_shape_and_device():
    d = synth.search_plan(max_templates=64)
    k = at.cache_key(d, "GB300")
    assert k == at.cache_key(d, "GB300")
    assert k != at.cache_key(d.replace(n_fft=1 << 21), "GB300")
    assert k != at.cache_key(d, "other")


def test_select_takes_fastest_within_tolerance():
    res = [dict(tuning="ref", ms=10.0, err=None), dict(tuning="fast_wrong", ms=5.0, err=1e-3),
           dict(tuning="fast_ok", ms=7.0, err=1e-6), dict(tuning="slow_ok", ms=9.0, err=0.0)]
    assert at.select(res, 2e-5)["tuning"] == "fast_ok"
    assert at.select(res[:1], 2e-5)["tuning"] == "ref"
    assert at.select([], 2e-5) is None


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert at.load_cache(path) == {}
    at.store_cache("k1", {"tuning": {"mode": 3, "log2_n1": 12, "chunk": 64, "knot_log2": 10}}, path)
    at.store_cache("k2", {"tuning": {"mode": 0, "log2_n1": 11, "chunk": 16, "knot_log2": 9}}, path)
    data = at.load_cache(path)
    assert data["k1"]["tuning"]["log2_n1"] == 12 and data["k2"]["tuning"]["mode"] == 0
