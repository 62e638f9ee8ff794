"""GB300 barycentric-resampling F-statistic.

Thin Python binding over ``libfstat.so`` (C ABI in ``include/fstat.h``).  The
functions below carry the names of the C entry points and only marshal
arguments: torch tensors provide device memory and streams, every step of
the computation runs in the library's CUDA kernels.

    plan = fstat_plan(desc)                  # desc: any object with the
                                             # fstat_plan_desc fields
    twoF = fstat_compute(plan, x_h, templates, gaps)
    fstat_status(plan)                       # raises on a device-side error
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (INJECTION_DTYPE, MODE_FUSED, MODE_PERSISTENT, MODE_PLAIN, MODE_SPLIT, NEAREST, PREC_FP32,
                   PREC_FP64, PREC_MIXED, SINC, TEMPLATE_DTYPE, WIN_LANCZOS, WIN_RECT)

__all__ = [
    "FstatError", "Plan", "fstat_plan", "fstat_compute", "fstat_compute_noalloc", "fstat_resample",
    "fstat_grad",
    "fstat_status", "fstat_destroy", "fstat_strerror", "fstat_template_nb", "pack_templates",
    "fstat_profile", "fstat_profile_read", "KERNEL_KINDS", "GraphRunner", "fstat_debug_stall", "fstat_topk", "fstat_stats",
    "fstat_inject", "pack_injections", "INJECTION_DTYPE", "fstat_sft_series", "fstat_sft_workspace",
    "fstat_sft_normalize", "fstat_sft_demod", "fstat_selftest_math",
    "NEAREST", "SINC", "WIN_RECT", "WIN_LANCZOS", "PREC_MIXED", "PREC_FP64", "PREC_FP32",
    "MODE_FUSED", "MODE_PLAIN", "MODE_PERSISTENT", "MODE_SPLIT", "TEMPLATE_DTYPE",
]


class FstatError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {fstat_strerror(code)} ({code})")


def fstat_strerror(code: int) -> str:
    return _lib.load().fstat_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != 0:
        raise FstatError(rc, where)


def _desc(d) -> _lib.PlanDesc:
    """fstat_plan_desc from any object carrying the same field names."""
    det = _lib.Detector(d.det.lat_rad, d.det.lon_rad, d.det.gamma_rad, d.det.radius_m)
    eph = _lib.Ephem(d.eph.au_m, d.eph.year_s, d.eph.sidereal_day_s, d.eph.obliquity_rad,
                     d.eph.orb_phase0, d.eph.sid_phase0)
    return _lib.PlanDesc(float(d.dt), float(d.t_start), int(d.n_data), float(d.f_het),
                         float(d.sigma2), int(d.n_fft), int(d.interp), int(d.taps),
                         int(d.window), int(d.precision), det, eph, int(d.max_templates))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def pack_templates(templates, device="cuda"):
    """Upload templates (a structured array with the fstat_template fields,
    or a sequence of dicts) as a device tensor of raw fstat_template
    records."""
    import torch
    arr = np.zeros(len(templates), dtype=TEMPLATE_DTYPE)
    for name in TEMPLATE_DTYPE.names:
        if isinstance(templates, np.ndarray) and templates.dtype.names:
            if name in templates.dtype.names:
                arr[name] = templates[name]
            elif name == "out_off":
                arr[name] = -1
        else:
            arr[name] = [t.get(name, -1 if name == "out_off" else 0) for t in templates]
    raw = torch.from_numpy(arr.view(np.uint8).copy())
    return raw.to(device) if device is not None else raw


def pack_injections(injections, device="cuda"):
    """Upload injections (a structured array with the fstat_injection
    fields) as a device tensor of raw fstat_injection records; returns
    (records, the longest span_len)."""
    import torch
    arr = np.zeros(len(injections), dtype=INJECTION_DTYPE)
    for name in INJECTION_DTYPE.names:
        arr[name] = injections[name]
    raw = torch.from_numpy(arr.view(np.uint8).copy())
    longest = int(arr["span_len"].max()) if len(arr) else 0
    return (raw.to(device) if device is not None else raw), longest


class Plan:
    """Owner of an fstat plan and of its torch-allocated workspace."""

    def __init__(self, desc, device=None):
        import torch
        self.lib = _lib.load()
        self.device = torch.device("cuda" if device is None else device)
        self.desc = desc
        h = ctypes.c_void_p()
        need = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            _check(self.lib.fstat_plan(ctypes.byref(h), ctypes.byref(_desc(desc)), ctypes.byref(need)),
                   "fstat_plan")
        self.handle = h
        self.workspace = None
        self._attach(need.value)

    def _attach(self, nbytes: int):
        import torch
        if self.workspace is not None and self.workspace.numel() >= nbytes:
            ws = self.workspace
        else:
            self.workspace = None
            ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=self.device)
        off = (-ws.data_ptr()) % 256
        self.workspace = ws
        _check(self.lib.fstat_set_workspace(self.handle, ctypes.c_void_p(ws.data_ptr() + off),
                                            ws.numel() - off), "fstat_set_workspace")

    def set_tuning(self, mode=MODE_SPLIT, log2_n1=0, cols=0, rows=0, chunk=0, knot_log2=0):
        need = ctypes.c_size_t()
        t = _lib.Tuning(mode, log2_n1, cols, rows, chunk, knot_log2)
        _check(self.lib.fstat_set_tuning(self.handle, ctypes.byref(t), ctypes.byref(need)),
               "fstat_set_tuning")
        self._attach(need.value)

    def set_band(self, q_lo: int, q_hi: int):
        """Write 2F only for bins q_lo <= q < q_hi (fstat_set_band)."""
        _check(self.lib.fstat_set_band(self.handle, int(q_lo), int(q_hi)), "fstat_set_band")

    def keep_lower_half(self):
        """The band-doubling remedy of Sec. V.B: of a search over twice the
        band it needs, keep the central half of the bins (|df| below a
        quarter of the sampling rate)."""
        n = int(self.desc.n_fft)
        self.set_band(n // 4, 3 * n // 4)

    def band(self) -> tuple:
        lo, hi = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.fstat_get_band(self.handle, ctypes.byref(lo), ctypes.byref(hi)), "fstat_get_band")
        return lo.value, hi.value

    def band_len(self) -> int:
        lo, hi = self.band()
        return hi - lo

    def tuning(self) -> dict:
        t = _lib.Tuning()
        _check(self.lib.fstat_get_tuning(self.handle, ctypes.byref(t)), "fstat_get_tuning")
        return {n: getattr(t, n) for n, _ in _lib.Tuning._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fstat_destroy(self.handle)
            self.handle = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fstat_plan(desc, device=None) -> Plan:
    return Plan(desc, device)


def fstat_destroy(plan: Plan):
    plan.close()


def _n_templates(templates) -> int:
    return templates.numel() // TEMPLATE_DTYPE.itemsize


def _gap_args(gaps):
    if gaps is None or gaps.numel() == 0:
        return ctypes.c_void_p(0), 0
    assert gaps.dtype.itemsize == 8 and gaps.is_cuda
    return _ptr(gaps), gaps.numel() // 2


def fstat_compute(plan: Plan, x_h, templates, gaps=None, twoF=None, stream=None):
    """2F for every template and bin of the plan's output band (float32,
    [n_templates * band length], the band being the whole n_fft unless
    set_band narrowed it; templates may carry their own offsets)."""
    import torch
    assert x_h.is_cuda and x_h.dtype == torch.complex64 and x_h.is_contiguous()
    n_t = _n_templates(templates)
    if twoF is None:
        twoF = torch.empty(n_t * plan.band_len(), dtype=torch.float32, device=x_h.device)
    g, ng = _gap_args(gaps)
    _check(plan.lib.fstat_compute(plan.handle, _ptr(x_h), _ptr(templates), n_t, g, ng,
                                  _ptr(twoF), _stream(stream)), "fstat_compute")
    return twoF


def fstat_compute_noalloc(desc, x_h, templates, gaps=None, twoF=None, stream=None):
    """fstat_compute without a plan or workspace: the library uses its own
    fixed scratch array (n_fft <= 2^20), for callers that cannot allocate
    device memory.  ``twoF`` (float32, at least n_templates * n_fft values)
    should be passed in by such callers.  The call runs on x_h's device, on
    that device's current stream unless ``stream`` is given; every tensor
    must live on that device."""
    import torch
    assert x_h.is_cuda and x_h.dtype == torch.complex64 and x_h.is_contiguous()
    dev = x_h.device
    lib = _lib.load()
    n_t = _n_templates(templates)
    need = n_t * int(desc.n_fft)
    for name, t in (("templates", templates), ("gaps", gaps), ("twoF", twoF)):
        if t is not None and t.device != dev:
            raise ValueError(f"fstat_compute_noalloc: {name} is on {t.device}, x_h on {dev}")
    if twoF is not None and (twoF.dtype != torch.float32 or not twoF.is_contiguous() or twoF.numel() < need):
        raise ValueError(f"fstat_compute_noalloc: twoF must be contiguous float32 with >= {need} values")
    with torch.cuda.device(dev):
        if twoF is None:
            twoF = torch.empty(need, dtype=torch.float32, device=dev)
        g, ng = _gap_args(gaps)
        s = _stream(torch.cuda.current_stream(dev) if stream is None else stream)
        _check(lib.fstat_compute_noalloc(ctypes.byref(_desc(desc)), _ptr(x_h), _ptr(templates), n_t, g, ng,
                                         _ptr(twoF), s), "fstat_compute_noalloc")
    return twoF


SELFTEST = {"sincospi_small": 0, "sincospif": 1, "expm2pi": 2, "sinc8_lanczos": 3, "sinc8_rect": 4}


def fstat_selftest_math(which: str, x, aux=None, stream=None):
    """The device math of the resampler on inputs x (float32, CUDA):
    a [n, 2] float32 tensor (fstat_selftest_math of the C ABI)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    out = torch.empty((x.numel(), 2), dtype=torch.float32, device=x.device)
    n_aux = 0 if aux is None else aux.numel()
    _check(_lib.load().fstat_selftest_math(SELFTEST[which], _ptr(x), x.numel(), _ptr(aux), n_aux, _ptr(out),
                                           _stream(stream)), "fstat_selftest_math")
    return out


def fstat_resample(plan: Plan, x_h, templates, gaps=None, stream=None):
    """Steps 1-5 only: (wa, wb, abcd) with wa, wb complex64 [n_t, n_fft]."""
    import torch
    n_t = _n_templates(templates)
    n = int(plan.desc.n_fft)
    wa = torch.empty((n_t, n), dtype=torch.complex64, device=x_h.device)
    wb = torch.empty_like(wa)
    abcd = torch.empty((n_t, 4), dtype=torch.float64, device=x_h.device)
    g, ng = _gap_args(gaps)
    _check(plan.lib.fstat_resample(plan.handle, _ptr(x_h), _ptr(templates), n_t, g, ng,
                                   _ptr(wa), _ptr(wb), _ptr(abcd), _stream(stream)), "fstat_resample")
    return wa, wb, abcd


def fstat_grad(plan: Plan, x_h, templates, df, gaps=None, stream=None):
    """2F at df (float64 [n_t]) and d2F/d(alpha, delta, f, fdot) ([n_t, 4])."""
    import torch
    n_t = _n_templates(templates)
    twoF = torch.empty(n_t, dtype=torch.float64, device=x_h.device)
    grad = torch.empty((n_t, 4), dtype=torch.float64, device=x_h.device)
    g, ng = _gap_args(gaps)
    df = df.to(device=x_h.device, dtype=torch.float64).contiguous()
    _check(plan.lib.fstat_grad(plan.handle, _ptr(x_h), _ptr(templates), _ptr(df), n_t, g, ng,
                               _ptr(twoF), _ptr(grad), _stream(stream)), "fstat_grad")
    return twoF, grad


KERNEL_KINDS = ("timemap", "resample", "fft_cols", "fft_rows", "grad_fwd", "grad_adj", "persistent", "sums")


def fstat_inject(plan: Plan, x_h, injections, max_span_len: int | None = None, stream=None):
    """Add the injections' signals to x_h (device complex64, in place).
    ``injections``: a structured array with the fstat_injection fields, or
    device records from ``pack_injections`` together with ``max_span_len``."""
    import torch
    assert x_h.is_cuda and x_h.dtype == torch.complex64 and x_h.is_contiguous()
    if isinstance(injections, np.ndarray):
        injections, longest = pack_injections(injections, device=x_h.device)
        max_span_len = longest if max_span_len is None else max_span_len
    if max_span_len is None:
        raise ValueError("max_span_len is needed with device records")
    n = injections.numel() // INJECTION_DTYPE.itemsize
    _check(plan.lib.fstat_inject(plan.handle, _ptr(injections), n, int(max_span_len), _ptr(x_h),
                                 _stream(stream)), "fstat_inject")
    return x_h


def _sft_desc(d) -> _lib.SftDesc:
    """fstat_sft_desc from any object carrying the same field names."""
    return _lib.SftDesc(int(d.sft_len), float(d.dt_raw), int(d.k_lo), int(d.n_bins), int(d.k_het),
                        int(d.band_bins), int(d.dirichlet_terms), int(d.median_window), float(d.tukey_frac),
                        int(d.edge_taper))


def fstat_sft_workspace(desc, n_sft: int) -> int:
    return int(_lib.load().fstat_sft_workspace(ctypes.byref(_sft_desc(desc)), int(n_sft)))


def fstat_sft_series(desc, sfts, t_sft, t_start: float, n_out: int, x_h=None, workspace=None, stream=None):
    """The heterodyned series from SFTs (steps 2-6 of Sec. III.B.7 on the
    GPU).  sfts: device complex64 [n_sft, n_bins]; t_sft: host start times
    (sequence of floats); returns x_h, device complex64 [n_out]."""
    import torch
    lib = _lib.load()
    assert sfts.is_cuda and sfts.dtype == torch.complex64 and sfts.is_contiguous()
    d = _sft_desc(desc)
    t = np.ascontiguousarray(np.asarray(t_sft, np.float64))
    n_sft = len(t)
    if x_h is None:
        x_h = torch.empty(int(n_out), dtype=torch.complex64, device=sfts.device)
    need = int(lib.fstat_sft_workspace(ctypes.byref(d), n_sft))
    if need == 0:
        raise FstatError(-1, "fstat_sft_workspace")
    if workspace is None or workspace.numel() < need + 256:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=sfts.device)
    off = (-workspace.data_ptr()) % 256
    _check(lib.fstat_sft_series(ctypes.byref(d), _ptr(sfts), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                n_sft, float(t_start), int(n_out), _ptr(x_h),
                                ctypes.c_void_p(workspace.data_ptr() + off), workspace.numel() - off,
                                _stream(stream)), "fstat_sft_series")
    return x_h


def fstat_sft_normalize(desc, sfts, out=None, stream=None):
    """Running-median noise normalisation of SFTs (device complex64
    [n_sft, n_bins]); returns the normalised copy."""
    import torch
    assert sfts.is_cuda and sfts.dtype == torch.complex64 and sfts.is_contiguous()
    out = torch.empty_like(sfts) if out is None else out
    _check(_lib.load().fstat_sft_normalize(ctypes.byref(_sft_desc(desc)), _ptr(sfts), sfts.shape[0], _ptr(out),
                                           _stream(stream)), "fstat_sft_normalize")
    return out


def fstat_sft_demod(plan: Plan, desc, sfts, t_sft, templates, q0: int, n_q: int, twoF=None, workspace=None,
                    stream=None):
    """SFT-domain demodulation 2F (the comparison method of Sec. IV.A) on
    bins q0 .. q0 + n_q - 1 of the plan's output grid.  sfts: normalised,
    device complex64 [n_sft, n_bins]; t_sft: device float64 [n_sft];
    templates: device records.  Returns float32 [n_t, n_q]."""
    import torch
    n_t = _n_templates(templates)
    n_sft = int(t_sft.numel())
    if twoF is None:
        twoF = torch.empty((n_t, int(n_q)), dtype=torch.float32, device=sfts.device)
    need = int(plan.lib.fstat_sft_demod_workspace(n_sft, n_t))
    if workspace is None or workspace.numel() < need + 256:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=sfts.device)
    off = (-workspace.data_ptr()) % 256
    _check(plan.lib.fstat_sft_demod(plan.handle, ctypes.byref(_sft_desc(desc)), _ptr(sfts), _ptr(t_sft), n_sft,
                                    _ptr(templates), n_t, int(q0), int(n_q), _ptr(twoF),
                                    ctypes.c_void_p(workspace.data_ptr() + off), workspace.numel() - off,
                                    _stream(stream)), "fstat_sft_demod")
    return twoF


def fstat_topk(two_f, band_len: int, k: int, n_rows: int | None = None, stream=None, val=None, bins=None):
    """Per-band top-k candidates of 2F rows (``two_f`` device float32 of
    n_rows x row_len, row_len = numel / n_rows): returns (values float32,
    bins int32), each [n_rows, row_len // band_len, k], descending, into
    ``val`` and ``bins`` when given (contiguous, at least that size)."""
    import torch
    lib = _lib.load()
    n_rows = 1 if n_rows is None else int(n_rows)
    row_len = two_f.numel() // n_rows
    n_bands = row_len // band_len if band_len else 0
    need = n_rows * n_bands * k
    if val is None:
        val = torch.empty((n_rows, n_bands, k), dtype=torch.float32, device=two_f.device)
    if bins is None:
        bins = torch.empty((n_rows, n_bands, k), dtype=torch.int32, device=two_f.device)
    if (val.dtype != torch.float32 or bins.dtype != torch.int32 or val.numel() < need or bins.numel() < need
            or not val.is_contiguous() or not bins.is_contiguous()
            or val.device != two_f.device or bins.device != two_f.device):
        raise ValueError(f"fstat_topk: val (float32) and bins (int32) need {need} contiguous values on {two_f.device}")
    _check(lib.fstat_topk(_ptr(two_f), n_rows, row_len, int(band_len), int(k), _ptr(val), _ptr(bins),
                          _stream(stream)), "fstat_topk")
    return val, bins


def fstat_stats(two_f, acc, thresholds=(), hist=None, bin_width: float = 1.0, stream=None):
    """Adds to ``acc`` (device float64, 3 + len(thresholds) values) the count
    of finite values of ``two_f`` (device float32), their sum, their sum of
    squares and the counts above each threshold, and to ``hist`` (device
    float64, one value per bin) the counts in bins of ``bin_width`` from 0,
    in one pass."""
    import torch
    lib = _lib.load()
    thr = (ctypes.c_float * max(1, len(thresholds)))(*[float(t) for t in thresholds])
    for name, t, dt in (("acc", acc, torch.float64), ("hist", hist, torch.float64)):
        if t is not None and (t.dtype != dt or not t.is_contiguous() or t.device != two_f.device):
            raise ValueError(f"fstat_stats: {name} must be contiguous float64 on {two_f.device}")
    if acc.numel() < 3 + len(thresholds):
        raise ValueError("fstat_stats: acc needs 3 + len(thresholds) values")
    assert two_f.is_cuda and two_f.dtype == torch.float32 and two_f.is_contiguous()
    n_bins = 0 if hist is None else hist.numel()
    _check(lib.fstat_stats(_ptr(two_f), two_f.numel(), thr, len(thresholds), float(bin_width), n_bins, _ptr(acc),
                           _ptr(hist) if hist is not None else None, _stream(stream)), "fstat_stats")
    return acc, hist


def fstat_profile(plan: Plan, enable: bool = True):
    """Enable/disable CUDA-event timing of every kernel launch."""
    _check(plan.lib.fstat_profile(plan.handle, int(bool(enable))), "fstat_profile")


def fstat_profile_read(plan: Plan) -> dict:
    """{kind: (milliseconds, launches)} since the last read (waits for the
    recorded events)."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    ln = (ctypes.c_int64 * n)()
    _check(plan.lib.fstat_profile_read(plan.handle, ms, ln, n), "fstat_profile_read")
    return {k: (ms[i], ln[i]) for i, k in enumerate(KERNEL_KINDS)}


def fstat_debug_stall(plan: Plan, template_index: int):
    """Arm the one-shot bounded-wait test hook of the persistent mode."""
    _check(plan.lib.fstat_debug_stall(plan.handle, int(template_index)), "fstat_debug_stall")


class GraphRunner:
    """A CUDA graph holding one fstat_compute call on fixed buffers; replay()
    reruns the whole batch (in persistent mode: the time map and one
    persistent launch) without host launch overhead.  The inputs are read
    from the same device tensors on every replay, so refill them in place."""

    def __init__(self, plan: Plan, x_h, templates, gaps=None, twoF=None, warmup: bool = True):
        import torch
        self.plan, self.x_h, self.templates, self.gaps = plan, x_h, templates, gaps
        n_t = _n_templates(templates)
        self.twoF = twoF if twoF is not None else torch.empty(n_t * plan.band_len(),
                                                              dtype=torch.float32, device=x_h.device)
        self.stream = torch.cuda.Stream(device=x_h.device)
        if warmup:   # first calls set kernel attributes outside the capture
            with torch.cuda.stream(self.stream):
                fstat_compute(plan, x_h, templates, gaps, self.twoF, stream=self.stream)
            self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            fstat_compute(plan, x_h, templates, gaps, self.twoF, stream=self.stream)

    def replay(self):
        """Replay on the runner's stream (synchronise it, or the device,
        before reading twoF)."""
        import torch
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        return self.twoF


def fstat_status(plan: Plan, stream=None, raise_error=True) -> int:
    rc = plan.lib.fstat_status(plan.handle, _stream(stream))
    if rc and raise_error:
        raise FstatError(rc, "device status")
    return rc


def fstat_template_nb(plan: Plan, templates_np) -> np.ndarray:
    """Resampled length N_b of each template (host computation)."""
    arr = np.ascontiguousarray(templates_np.astype(TEMPLATE_DTYPE) if templates_np.dtype != TEMPLATE_DTYPE
                               else templates_np)
    out = np.zeros(len(arr), dtype=np.int64)
    _check(plan.lib.fstat_template_nb(plan.handle, arr.ctypes.data_as(ctypes.POINTER(_lib.Template)),
                                      len(arr), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "fstat_template_nb")
    return out
