"""The C ABI without a GPU: the library builds, exports every function the
header declares, its structures have the header's layout, and host-side
argument checks answer before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fstat.h")


@pytest.fixture(scope="module")
def lib():
    from paper_0912_4255_gb300 import build
    build.build()
    from paper_0912_4255_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fstat_[a-z_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("fstat_plan", "fstat_set_workspace", "fstat_resample", "fstat_compute",
              "fstat_grad", "fstat_status", "fstat_destroy", "fstat_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (fstat_\w+)", out.stdout))
    for n in declared_functions():
        assert n in exported, n
        assert getattr(lib, n) is not None


def _c_layout():
    """sizeof/offsetof of the header structures as the C compiler sees them."""
    from paper_0912_4255_gb300 import _lib
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for cname, cls in (("fstat_detector", _lib.Detector), ("fstat_ephem", _lib.Ephem),
                       ("fstat_plan_desc", _lib.PlanDesc), ("fstat_template", _lib.Template),
                       ("fstat_tuning", _lib.Tuning), ("fstat_injection", _lib.Injection),
                       ("fstat_sft_desc", _lib.SftDesc)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", c, "-o", exe], check=True)
        return subprocess.run([exe], capture_output=True, text=True, check=True).stdout


def test_struct_layouts_match_header():
    from paper_0912_4255_gb300 import _lib
    got = {}
    for line in _c_layout().splitlines():
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in (("fstat_detector", _lib.Detector), ("fstat_ephem", _lib.Ephem),
                       ("fstat_plan_desc", _lib.PlanDesc), ("fstat_template", _lib.Template),
                       ("fstat_tuning", _lib.Tuning), ("fstat_injection", _lib.Injection),
                       ("fstat_sft_desc", _lib.SftDesc)):
        assert got[(cname, "size")] == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_strerror(lib):
    for code in range(-7, 1):
        assert lib.fstat_strerror(code)
    assert b"unknown" in lib.fstat_strerror(-99)


def _desc(**kw):
    import synth
    from paper_0912_4255_gb300 import _desc as mk
    return mk(synth.tiny_plan(**kw))


@pytest.mark.parametrize("kw,code", [
    (dict(dt=0.0), -1), (dict(sigma2=-1.0), -1), (dict(n_data=1), -1),
    (dict(n_fft=1000), -2), (dict(n_fft=1 << 25), -2), (dict(interp=7), -1),
    (dict(interp=1, taps=3), -6), (dict(precision=9), -1), (dict(window=5), -1),
])
def test_plan_rejects_bad_descriptors_on_the_host(lib, kw, code):
    h = ctypes.c_void_p()
    need = ctypes.c_size_t()
    d = _desc(**kw)
    assert lib.fstat_plan(ctypes.byref(h), ctypes.byref(d), ctypes.byref(need)) == code
    assert not h.value


def test_null_arguments(lib):
    assert lib.fstat_plan(None, None, None) == -1
    assert lib.fstat_status(None, None) == -1
    assert lib.fstat_compute(None, None, None, 0, None, 0, None, None) == -1
    lib.fstat_destroy(None)


def test_inject_rejects_bad_arguments_on_the_host(lib):
    """fstat_inject checks its plan, pointers and sizes before any launch."""
    assert lib.fstat_inject(None, None, 0, 0, None, None) == -1               # no plan
    assert lib.fstat_inject(None, None, 1, 86400, None, None) == -1


def test_sft_front_end_checks_its_descriptor_on_the_host(lib):
    """fstat_sft_workspace / fstat_sft_series validate the descriptor before
    any device work (no GPU needed)."""
    import synth
    from paper_0912_4255_gb300 import _sft_desc
    good = synth.SftDesc(sft_len=2048, k_lo=344, n_bins=112, k_het=400, band_bins=64, dirichlet_terms=16)
    assert lib.fstat_sft_workspace(ctypes.byref(_sft_desc(good)), 10) > 0
    for bad, code in [(dict(band_bins=63), -1), (dict(median_window=10), -1), (dict(dt_raw=0.0), -1),
                      (dict(tukey_frac=1.5), -1), (dict(k_lo=360), -2), (dict(n_bins=90), -2),
                      (dict(dirichlet_terms=-1), -1)]:
        d = _sft_desc(good.replace(**bad))
        assert lib.fstat_sft_workspace(ctypes.byref(d), 10) == 0
        assert lib.fstat_sft_series(ctypes.byref(d), None, None, 0, 0.0, 0, None, None, 0, None) == code
    d = _sft_desc(good)
    assert lib.fstat_sft_series(ctypes.byref(d), None, None, 0, 0.0, 0, None, None, 0, None) == -1   # no output


def test_injection_records_match_the_struct():
    import synth
    from paper_0912_4255_gb300 import _lib
    assert synth.INJECTION_DTYPE == _lib.INJECTION_DTYPE
    r = synth.random_injection_records(3, 1, 0.01, 0.5, 1000, span_start0=7)
    assert list(r["span_start"]) == [7, 1007, 2007] and np.all(r["span_len"] == 1000)
    assert np.all(np.abs(r["delta"]) <= np.pi / 2) and np.all(np.abs(r["cosi"]) <= 1)


def test_topk_rejects_bad_arguments_on_the_host(lib):
    """fstat_topk checks its sizes and pointers before any launch."""
    p = 4096          # a 16-byte aligned stand-in pointer (never dereferenced)
    assert lib.fstat_topk(None, 1, 4096, 2048, 4, p, p, None) == -1          # null input
    assert lib.fstat_topk(p + 4, 1, 4096, 2048, 4, p, p, None) == -1         # not 16-byte aligned
    assert lib.fstat_topk(p, 1, 4096, 2048, 0, p, p, None) == -1             # k < 1
    assert lib.fstat_topk(p, 1, 4096, 2048, 65, p, p, None) == -1            # k > 64
    assert lib.fstat_topk(p, 1, 4096, 1024, 4, p, p, None) == -1             # band below 2048
    assert lib.fstat_topk(p, 1, 6144, 4096, 4, p, p, None) == -1             # band does not divide
    assert lib.fstat_topk(p, 70000, 4096, 2048, 4, p, p, None) == -2         # too many rows
    assert lib.fstat_topk(p, 0, 4096, 2048, 4, p, p, None) == 0              # nothing to do


def test_stats_rejects_bad_arguments_on_the_host(lib):
    """fstat_stats checks its sizes and pointers before any launch."""
    import ctypes
    p = 4096                                   # a 16-byte aligned stand-in pointer (never dereferenced)
    thr = (ctypes.c_float * 4)(10.0, 20.0, 30.0, 40.0)
    assert lib.fstat_stats(p, 0, thr, 3, 1.0, 40, p, p, None) == 0           # nothing to do
    assert lib.fstat_stats(None, 8, thr, 3, 1.0, 40, p, p, None) == -1       # null input
    assert lib.fstat_stats(p + 4, 8, thr, 3, 1.0, 40, p, p, None) == -1      # not 16-byte aligned
    assert lib.fstat_stats(p, 8, thr, 5, 1.0, 40, p, p, None) == -1          # more than 4 thresholds
    assert lib.fstat_stats(p, 8, thr, 3, 1.0, 257, p, p, None) == -1         # more than 256 bins
    assert lib.fstat_stats(p, 8, thr, 3, 0.0, 40, p, p, None) == -1          # bin width 0
    assert lib.fstat_stats(p, 8, thr, 3, 1.0, 40, p, None, None) == -1       # bins without hist
    assert lib.fstat_stats(p, 8, thr, 3, 1.0, 40, None, p, None) == -1       # no accumulators
    assert lib.fstat_stats(p, -1, thr, 3, 1.0, 40, p, p, None) == -1         # negative count
