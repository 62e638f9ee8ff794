"""SFT-domain demodulation F-statistic (FP64, test oracle): the earlier
method the paper compares against (Sec. IV.A), re-derived from the paper's
own equations.

TEST INFRASTRUCTURE: only tests/, the smoke check and the bench's CPU
baseline may use this module; the library never does.

Derivation.  Eq. 7 demodulates the data with the template phase,
F_a = sum_t a(t) x(t) e^{-i Phi(t)} (e^{-i Phi}: reading G1), Phi(t) =
2 pi (f tau + fdot tau^2 / 2 + fddot tau^3 / 6), tau = t - t_s + t_m(t)
(Eq. 4, absolute frequency f).  Within SFT alpha (start t_alpha, N raw
samples, length T, midpoint tm_alpha) take the phase as linear and a, b as
constant at the midpoint:
  Phi(t) ~ Phi_alpha + 2 pi fhat_alpha (t - tm_alpha),
  fhat_alpha = (f + fdot tau + fddot tau^2 / 2)(1 + dt_m/dt) at tm_alpha.
Writing the samples through the SFT's inverse DFT (Eq. e3) the sum over the
SFT's samples becomes e^{-i Phi_alpha} e^{i pi kappa_alpha} times the SFT
evaluated at the fractional bin kappa_alpha = fhat_alpha T, which the
Dirichlet kernel of Eq. e9 interpolates:
  X(kappa) = sum_k X_{alpha,k} P(kappa - k),
  P = sin y / y - i (1 - cos y) / y,  y = 2 pi (kappa - k)   (P = 1 at y = 0),
truncated to k* - dk .. k* + dk, k* = floor(kappa).  So
  F_a = sum_alpha a_alpha e^{-2 pi i (Phi_alpha / 2 pi - kappa_alpha / 2)} X_alpha(kappa_alpha),
F_b the same with b_alpha, and for normalised SFTs (E|X^|^2 = 1, so that
the interpolated bins have unit noise variance)
  A = sum a_alpha^2, B = sum b_alpha^2, C = sum a_alpha b_alpha, D = AB - C^2,
  2F = 2 (B |F_a|^2 + A |F_b|^2 - 2 C Re F_a F_b*) / D,
which has mean 4 in noise (the normalisation of Eq. LALDemodFstat).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry


def _frac(x):
    return x - np.floor(x)


def sft_midpoint_terms(plan, sd, t_sft, alpha, delta, fdot=0.0, fddot=0.0):
    """Per SFT: tau, dt_m/dt and a, b at the SFT midpoints."""
    T = sd.sft_len * sd.dt_raw
    tm_ = np.asarray(t_sft, np.float64) + T / 2.0
    t_m = geometry.roemer_delay(tm_, alpha, delta, plan.det, plan.eph)
    rate = geometry.roemer_rate(tm_, alpha, delta, plan.det, plan.eph)
    a, b = geometry.beam_ab(tm_, alpha, delta, plan.det, plan.eph)[:2]
    tau = tm_ - plan.t_start + t_m
    return tau, rate, a, b


def two_f(X, sd, plan, t_sft, alpha, delta, f, fdot=0.0, fddot=0.0):
    """2F of normalised SFT bins X (n_sft, n_bins; stored bins k_lo ..) at
    the absolute frequencies f (array), for one sky position and spindown."""
    T = sd.sft_len * sd.dt_raw
    tau, rate, a, b = sft_midpoint_terms(plan, sd, t_sft, alpha, delta, fdot, fddot)
    A, B, C = np.sum(a * a), np.sum(b * b), np.sum(a * b)
    D = A * B - C * C
    f = np.atleast_1d(np.asarray(f, np.float64))
    out = np.empty(f.size)
    for i, fi in enumerate(f):
        fhat = (fi + fdot * tau + 0.5 * fddot * tau ** 2) * (1.0 + rate)
        kappa = fhat * T
        cyc = _frac(fi * tau) + _frac(0.5 * fdot * tau ** 2) + _frac(fddot * tau ** 3 / 6.0)
        rot = np.exp(-2j * math.pi * (cyc - 0.5 * kappa))
        Fa = Fb = 0.0j
        for al in range(len(tau)):
            ks = int(math.floor(kappa[al]))
            s = 0.0j
            for k in range(ks - sd.dirichlet_terms, ks + sd.dirichlet_terms + 1):
                y = 2.0 * math.pi * (kappa[al] - k)
                P = 1.0 + 0.0j if y == 0.0 else complex(math.sin(y) / y, -(1.0 - math.cos(y)) / y)
                s += X[al, k - sd.k_lo] * P
            Fa += a[al] * rot[al] * s
            Fb += b[al] * rot[al] * s
        out[i] = 2.0 * (B * abs(Fa) ** 2 + A * abs(Fb) ** 2 - 2.0 * C * (Fa * np.conj(Fb)).real) / D
    return out
