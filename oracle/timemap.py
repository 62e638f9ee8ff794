"""Barycentric time grid and its inverse map (FP64, test oracle).

Eq. 11: t_b = t + t_m(t).  Eq. 21 and the procedure of Sec. III.A.2 (step 3):
the resampled series lives on a uniform grid t_b^k in the barycentric frame,
and the detector times T^k(t_b^k) that map onto it are needed to interpolate
the detector-frame data.

The paper does not say how the grid starts or how the inverse is computed.
Readings used here:

* grid: t_b^k = t_b(t_s) + k dt, k = 0 .. N_b - 1, with
  N_b = floor((t_b(t_e) - t_b(t_s)) / dt) + 1, where t_s and t_e are the times
  of the first and last sample of the template's span;
* inverse: fixed-point iteration T <- t_b^k - t_m(T) from
  T_0 = t_b^k - t_m(t_b^k).  The map contracts by |dt_m/dt| <~ 1e-4
  (Eq. 11c), so each iteration gains four decimal digits.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import roemer_delay


def span_times(tmpl, plan):
    """Times of the first and last sample of a template's span."""
    t_s = plan.t_start + int(tmpl["span_start"]) * plan.dt
    t_e = plan.t_start + (int(tmpl["span_start"]) + int(tmpl["span_len"]) - 1) * plan.dt
    return t_s, t_e


def grid(tmpl, plan):
    """(t_b0, N_b): start of the uniform barycentric grid and its length."""
    a, d = float(tmpl["alpha"]), float(tmpl["delta"])
    t_s, t_e = span_times(tmpl, plan)
    tb_s = t_s + float(roemer_delay(t_s, a, d, plan.det, plan.eph))
    tb_e = t_e + float(roemer_delay(t_e, a, d, plan.det, plan.eph))
    n_b = int(math.floor((tb_e - tb_s) / plan.dt)) + 1
    return tb_s, n_b


def inverse_map(t_b, alpha, delta, plan, iters: int = 6):
    """Detector times T with T + t_m(T) = t_b (fixed-point iteration)."""
    t_b = np.asarray(t_b, dtype=np.float64)
    T = t_b - roemer_delay(t_b, alpha, delta, plan.det, plan.eph)
    for _ in range(iters):
        T = t_b - roemer_delay(T, alpha, delta, plan.det, plan.eph)
    return T


def resample_times(tmpl, plan):
    """t_b^k and T^k for every grid point of a template, plus N_b."""
    tb0, n_b = grid(tmpl, plan)
    tb = tb0 + np.arange(n_b, dtype=np.float64) * plan.dt
    T = inverse_map(tb, float(tmpl["alpha"]), float(tmpl["delta"]), plan)
    return tb, T, n_b
