"""Autotuner of the library's execution shape.

The batched path has a few free choices that do not change what is computed:
the execution mode (split, fused, persistent), the factorisation N = N1 N2 of
the four-step FFT (``log2_n1``), the templates per internal batch (``chunk``)
and the knot spacing of the time map (``knot_log2``).  ``autotune`` times
``fstat_compute`` under each candidate on a probe batch of the caller's own
inputs, keeps only candidates whose 2F reproduces the default tuning's to
within ``tol`` (R15 metric: max |a - b| / max(b, 4)), and returns the fastest.
Results are cached per GPU model and plan shape in a JSON file.

Everything here is host-side orchestration: the timed work is the library's
CUDA kernels.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from ._lib import MODE_FUSED, MODE_PERSISTENT, MODE_SPLIT, PREC_FP64

__all__ = ["candidates", "cache_key", "load_cache", "store_cache", "autotune", "apply_cached"]

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fstat_gb300", "tune.json")


def _log2(n: int) -> int:
    return int(n).bit_length() - 1


def default_knot_log2(f_het: float, dt: float) -> int:
    """The library's default knot spacing of the time map (log2 of grid
    points per knot): 11 while |f_het dt| <= 50 and dt <= 0.5 s, 10 up to
    100, 9 beyond; the autotuner tries the next denser spacing."""
    c = abs(f_het * dt)
    return 11 if (c <= 50.0 and dt <= 0.5) else (10 if c <= 100.0 else 9)


def candidates(desc, modes=None, chunks=None, knots=True):
    """Tunings worth timing for a plan: every valid first-pass length
    (2^6 <= N1, N2 <= 2^12) in split mode, the default shape in the other
    modes, a smaller chunk, and the next denser knot spacing (more accurate,
    never sparser).  Zeros mean "the library's default"."""
    L = _log2(desc.n_fft)
    lo, hi = max(6, L - 12), min(12, L - 6)
    if modes is None:
        modes = [MODE_SPLIT, MODE_FUSED]
        if desc.precision != PREC_FP64 and desc.max_templates <= 65535:
            modes.append(MODE_PERSISTENT)
    out = [dict(mode=MODE_SPLIT)]
    for m in modes:
        shapes = range(lo, hi + 1) if m == MODE_SPLIT else [0]
        for l1 in shapes:
            t = dict(mode=m, log2_n1=l1)
            if t not in out:
                out.append(t)
    if chunks:
        for c in chunks:
            out.append(dict(mode=MODE_SPLIT, chunk=int(c)))
    if knots:
        out.append(dict(mode=MODE_SPLIT, knot_log2=default_knot_log2(desc.f_het, desc.dt) - 1))
    return out


def cache_key(desc, device_name: str) -> str:
    """Stable key of the plan fields that change which tuning is fastest."""
    fields = (device_name, int(desc.n_data), int(desc.n_fft), float(desc.dt), float(desc.f_het),
              int(desc.interp), int(desc.taps), int(desc.window), int(desc.precision),
              int(desc.max_templates))
    return hashlib.sha1(repr(fields).encode()).hexdigest()[:16]


def load_cache(path: str | None = None) -> dict:
    path = path or os.environ.get("FSTAT_TUNE_CACHE", DEFAULT_CACHE)
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, entry: dict, path: str | None = None):
    path = path or os.environ.get("FSTAT_TUNE_CACHE", DEFAULT_CACHE)
    data = load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def r15(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(b, 4.0)))


def select(results, tol: float):
    """The fastest accepted result: results are dicts with 'ms' and 'err'
    (None for the reference); a candidate is accepted when err <= tol."""
    ok = [r for r in results if r.get("err") is None or r["err"] <= tol]
    return min(ok, key=lambda r: r["ms"]) if ok else None


def autotune(plan, x_h, templates, gaps=None, *, cands=None, repeats: int = 3, tol: float = 2e-5,
             cache: str | None = None, use_cache: bool = True, apply: bool = True, log=None) -> dict:
    """Time fstat_compute on (x_h, templates, gaps) under each candidate
    tuning and set the fastest accepted one on ``plan``.  Returns
    {"tuning": ..., "ms": ..., "results": [...]}.  The probe batch should be
    representative (a full batch of the search); its outputs are compared
    with the default tuning's."""
    import torch
    from . import _n_templates, fstat_compute, fstat_status

    dev_name = torch.cuda.get_device_name(plan.device)
    key = cache_key(plan.desc, dev_name)
    if use_cache:
        hit = load_cache(cache).get(key)
        if hit:
            if apply:
                plan.set_tuning(**hit["tuning"])
            return dict(hit, cached=True)
    cands = cands if cands is not None else candidates(plan.desc)
    n_t = _n_templates(templates)
    out = torch.empty(n_t * int(plan.desc.n_fft), dtype=torch.float32, device=plan.device)
    stream = torch.cuda.Stream(device=plan.device)
    ref = None
    results = []
    for t in cands:
        try:
            plan.set_tuning(**t)
        except Exception as e:          # a shape the library rejects for this plan
            results.append(dict(tuning=t, ms=float("inf"), err=float("inf"), skipped=str(e)))
            continue
        with torch.cuda.stream(stream):
            fstat_compute(plan, x_h, templates, gaps, out, stream=stream)      # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(repeats):
                fstat_compute(plan, x_h, templates, gaps, out, stream=stream)
            e1.record(stream)
        stream.synchronize()
        if fstat_status(plan, stream, raise_error=False) != 0:
            results.append(dict(tuning=t, ms=float("inf"), err=float("inf"), skipped="device status"))
            continue
        ms = e0.elapsed_time(e1) / repeats
        got = out.cpu().numpy()
        if ref is None:
            ref = got.copy()
            err = None
        else:
            err = r15(got, ref)
        entry = dict(tuning=plan.tuning(), ms=ms, err=err)
        results.append(entry)
        if log:
            log(entry)
    best = select(results, tol)
    if best is None:
        raise RuntimeError("no tuning could be timed")
    tuning = {k: int(best["tuning"][k]) for k in ("mode", "log2_n1", "chunk", "knot_log2")}
    entry = dict(tuning=tuning, ms=best["ms"], device=dev_name)
    if use_cache:
        store_cache(key, entry, cache)
    if apply:
        plan.set_tuning(**tuning)
    return dict(entry, results=results, cached=False)


def apply_cached(plan, cache: str | None = None) -> bool:
    """Set a cached tuning on ``plan`` if one exists for its GPU and shape."""
    import torch
    hit = load_cache(cache).get(cache_key(plan.desc, torch.cuda.get_device_name(plan.device)))
    if hit:
        plan.set_tuning(**hit["tuning"])
        return True
    return False
