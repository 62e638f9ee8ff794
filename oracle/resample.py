"""Interpolation of the detector-frame series at T^k and the gap mask
(FP64, test oracle).

Sec. III.A.2, step 4: z(T^k(t_b^k)) is obtained from the regularly sampled
z(t^k) by interpolation; the paper does not fix the interpolator.  Sec. V.B
notes the low-pass loss of interpolation.  Readings used here:

* fractional index u_k = (T^k - t_start) / dt;
* nearest neighbour: source j = floor(u_k + 1/2);
* K-tap windowed sinc (a truncated Dirichlet/sinc interpolator): sum over
  j = floor(u) - K/2 + 1 .. floor(u) + K/2 of
  x[j] sinc(u - j) W((u - j)/(K/2)), sinc(x) = sin(pi x)/(pi x),
  W = 1 (rectangular, plain truncation) or W(y) = sinc(y) (Lanczos);
* taps outside the template's span or inside a gap contribute zero
  (Sec. III.B, "Gaps in the data": gaps act like zero padding);
* mask m_k = 1 iff the nearest-neighbour source sample lies inside the span
  and outside every gap; the resampled value is multiplied by m_k.
"""
from __future__ import annotations

import numpy as np

NEAREST, SINC = 0, 1
WIN_RECT, WIN_LANCZOS = 0, 1


def valid_samples(n_data, span_start, span_len, gaps):
    """Boolean validity of every data sample for one template."""
    v = np.zeros(n_data, dtype=bool)
    v[span_start:span_start + span_len] = True
    for s, e in np.asarray(gaps, dtype=np.int64).reshape(-1, 2):
        v[s:e] = False
    return v


def fractional_index(T, plan):
    return (np.asarray(T, dtype=np.float64) - plan.t_start) / plan.dt


def nn_source(u):
    return np.floor(u + 0.5).astype(np.int64)


def mask(u, valid):
    """m_k from the nearest-neighbour source sample."""
    j = nn_source(u)
    ok = (j >= 0) & (j < valid.size)
    m = np.zeros(u.shape, dtype=np.float64)
    m[ok] = valid[j[ok]]
    return m


def sinc(x):
    return np.sinc(x)  # sin(pi x)/(pi x) with sinc(0) = 1


def interpolate(x, u, valid, interp, taps=8, window=WIN_LANCZOS):
    """z(u_k) from the samples x[j] (complex), zero outside ``valid``."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    xv = np.where(valid, x, 0.0)
    if interp == NEAREST:
        j = nn_source(u)
        ok = (j >= 0) & (j < n)
        out = np.zeros(u.shape, dtype=np.complex128)
        out[ok] = xv[j[ok]]
        return out
    if interp != SINC:
        raise ValueError("unknown interpolation kind")
    half = taps // 2
    base = np.floor(u).astype(np.int64)
    out = np.zeros(u.shape, dtype=np.complex128)
    for i in range(taps):
        j = base - half + 1 + i
        d = u - j
        w = sinc(d)
        if window == WIN_LANCZOS:
            w = w * sinc(d / half)
        ok = (j >= 0) & (j < n)
        out[ok] += xv[j[ok]] * w[ok]
    return out


def nn_tie_margin(u):
    """Distance of the fractional indices from a nearest-neighbour rounding
    tie (|frac(u) - 1/2|); the NN decision is unique where this margin
    exceeds the arithmetic error of u."""
    f = u - np.floor(u)
    return float(np.min(np.abs(f - 0.5))) if u.size else 1.0
