"""ctypes declarations of ``include/fstat.h`` and the loader of libfstat.so.

Pure marshalling: the structures mirror the header field by field; every
computation happens in the CUDA library.  There is no fallback: if the
library is missing the import of the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfstat.so")

FSTAT_OK, FSTAT_EINVAL, FSTAT_ERANGE, FSTAT_ENOMEM = 0, -1, -2, -3
FSTAT_ECUDA, FSTAT_ETIMEOUT, FSTAT_ENOTSUP, FSTAT_ENOWS = -4, -5, -6, -7
NEAREST, SINC = 0, 1
WIN_RECT, WIN_LANCZOS = 0, 1
PREC_MIXED, PREC_FP64, PREC_FP32 = 0, 1, 2
MODE_FUSED, MODE_PLAIN, MODE_PERSISTENT, MODE_SPLIT = 0, 1, 2, 3

c_double, c_int64, c_int32, c_void_p = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p


class Detector(ctypes.Structure):
    _fields_ = [("lat_rad", c_double), ("lon_rad", c_double), ("gamma_rad", c_double),
                ("radius_m", c_double)]


class Ephem(ctypes.Structure):
    _fields_ = [("au_m", c_double), ("year_s", c_double), ("sidereal_day_s", c_double),
                ("obliquity_rad", c_double), ("orb_phase0", c_double), ("sid_phase0", c_double)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("dt", c_double), ("t_start", c_double), ("n_data", c_int64),
                ("f_het", c_double), ("sigma2", c_double), ("n_fft", c_int64),
                ("interp", c_int32), ("taps", c_int32), ("window", c_int32),
                ("precision", c_int32), ("det", Detector), ("eph", Ephem),
                ("max_templates", c_int64)]


class Template(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("delta", c_double), ("fdot", c_double),
                ("span_start", c_int64), ("span_len", c_int64),
                ("gap_off", c_int64), ("n_gaps", c_int64),
                ("n_fft", c_int64), ("out_off", c_int64), ("fddot", c_double)]


class Injection(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("delta", c_double), ("psi", c_double), ("cosi", c_double),
                ("phi0", c_double), ("h0", c_double), ("df", c_double), ("fdot", c_double),
                ("fddot", c_double), ("span_start", c_int64), ("span_len", c_int64)]


class SftDesc(ctypes.Structure):
    _fields_ = [("sft_len", c_int64), ("dt_raw", c_double), ("k_lo", c_int64), ("n_bins", c_int64),
                ("k_het", c_int64), ("band_bins", c_int64), ("dirichlet_terms", ctypes.c_int32),
                ("median_window", ctypes.c_int32), ("tukey_frac", c_double), ("edge_taper", c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("log2_n1", c_int32), ("cols", c_int32),
                ("rows", c_int32), ("chunk", c_int32), ("knot_log2", c_int32)]


# numpy view of fstat_template (same layout as the C struct)
TEMPLATE_DTYPE = np.dtype([(n, np.float64 if t is c_double else np.int64)
                           for n, t in Template._fields_])
assert TEMPLATE_DTYPE.itemsize == ctypes.sizeof(Template)
# numpy view of fstat_injection
INJECTION_DTYPE = np.dtype([(n, np.float64 if t is c_double else np.int64)
                            for n, t in Injection._fields_])
assert INJECTION_DTYPE.itemsize == ctypes.sizeof(Injection)

SYMBOLS = {
    "fstat_plan": (ctypes.c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(PlanDesc),
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "fstat_set_tuning": (ctypes.c_int, [c_void_p, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_size_t)]),
    "fstat_get_tuning": (ctypes.c_int, [c_void_p, ctypes.POINTER(Tuning)]),
    "fstat_set_workspace": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_size_t]),
    "fstat_template_nb": (ctypes.c_int, [c_void_p, ctypes.POINTER(Template), c_int64,
                                         ctypes.POINTER(c_int64)]),
    "fstat_resample": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                      c_void_p, c_void_p, c_void_p, c_void_p]),
    "fstat_compute": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                     c_void_p, c_void_p]),
    "fstat_grad": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                  c_int64, c_void_p, c_void_p, c_void_p]),
    "fstat_compute_noalloc": (ctypes.c_int, [ctypes.POINTER(PlanDesc), c_void_p, c_void_p, c_int64,
                                             c_void_p, c_int64, c_void_p, c_void_p]),
    "fstat_debug_stall": (ctypes.c_int, [c_void_p, c_int64]),
    "fstat_selftest_math": (ctypes.c_int, [ctypes.c_int, c_void_p, c_int64, c_void_p, c_int64, c_void_p,
                                           c_void_p]),
    "fstat_topk": (ctypes.c_int, [c_void_p, c_int64, c_int64, c_int64, ctypes.c_int, c_void_p, c_void_p,
                                  c_void_p]),
    "fstat_stats": (ctypes.c_int, [c_void_p, c_int64, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_float,
                                   ctypes.c_int, c_void_p, c_void_p, c_void_p]),
    "fstat_set_band": (ctypes.c_int, [c_void_p, c_int64, c_int64]),
    "fstat_get_band": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)]),
    "fstat_sft_workspace": (ctypes.c_size_t, [ctypes.POINTER(SftDesc), c_int64]),
    "fstat_sft_series": (ctypes.c_int, [ctypes.POINTER(SftDesc), c_void_p, ctypes.POINTER(c_double), c_int64,
                                        c_double, c_int64, c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "fstat_sft_normalize": (ctypes.c_int, [ctypes.POINTER(SftDesc), c_void_p, c_int64, c_void_p, c_void_p]),
    "fstat_sft_demod_workspace": (ctypes.c_size_t, [c_int64, c_int64]),
    "fstat_sft_demod": (ctypes.c_int, [c_void_p, ctypes.POINTER(SftDesc), c_void_p, c_void_p, c_int64, c_void_p,
                                       c_int64, c_int64, c_int64, c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "fstat_inject": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p]),
    "fstat_profile": (ctypes.c_int, [c_void_p, ctypes.c_int]),
    "fstat_profile_read": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64),
                                          ctypes.c_int]),
    "fstat_status": (ctypes.c_int, [c_void_p, c_void_p]),
    "fstat_destroy": (None, [c_void_p]),
    "fstat_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfstat.so (built by ``paper_0912_4255_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_0912_4255_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
