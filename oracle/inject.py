"""Signal injection and optimal SNR (FP64, test oracle).

Strain h = F_+ h_+ + F_x h_x (Eq. 1) with h_+ = A_+ cos Psi,
h_x = A_x sin Psi, A_+ = h0 (1 + cos^2 iota)/2, A_x = h0 cos iota, and the
phase Psi(t) = Phi_0 + 2 pi (f tau + fdot tau^2 / 2 + fddot tau^3 / 6) with
tau = t - t_start + t_m(t) (Eq. 4 to s = 2 written in barycentric time).
The detector series handed to the search is the heterodyned, band-limited
complex series x_h = x exp(-2 pi i f_h (t - t_start)) (Sec. III.A.1); of the
real signal only its positive-frequency half survives the low-pass, so

  x_h[n] = 1/2 (F_+ A_+ - i F_x A_x) exp(i [Psi(t_n) - 2 pi f_h (t_n - t_start)]).

The antenna functions come from the detector-tensor form (independent of the
closed form used by the search), so a search that recovers rho^2 also checks
the closed form.

Optimal SNR for complex data with E|n|^2 = sigma^2:
rho^2 = 2 sum |s_n|^2 / sigma^2 = sum (F_+^2 A_+^2 + F_x^2 A_x^2) / (2 sigma^2),
the non-centrality of 2F (Sec. IV.B).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, resample


def _frac(x):
    return x - np.floor(x)


def signal(inj, plan, n_data=None, h0=None, valid=None):
    """Complex heterodyned signal of one injection at every data sample
    (zero where ``valid`` is False)."""
    n_data = int(n_data or plan.n_data)
    h0 = float(h0 if h0 is not None else (inj.h0 if inj.h0 is not None else 1.0))
    t = plan.t_start + np.arange(n_data) * plan.dt
    tm = geometry.roemer_delay(t, inj.alpha, inj.delta, plan.det, plan.eph)
    tau = t - plan.t_start + tm
    Fp, Fx = geometry.antenna_tensor(t, inj.alpha, inj.delta, inj.psi, plan.det, plan.eph)
    Ap = h0 * (1.0 + inj.cosi ** 2) / 2.0
    Ax = h0 * inj.cosi
    f = plan.f_het + inj.df
    # Psi - 2 pi f_h (t - t_start) in cycles, reduced before exponentiation:
    # f tau - f_h (t - t_start) = f_h t_m + df tau
    cyc = (_frac(plan.f_het * tm) + _frac(inj.df * tau)
           + _frac(0.5 * inj.fdot * tau * tau) + _frac(getattr(inj, "fddot", 0.0) * tau ** 3 / 6.0)
           + inj.phi0 / (2 * math.pi))
    s = 0.5 * (Fp * Ap - 1j * Fx * Ax) * np.exp(2j * np.pi * _frac(cyc))
    if valid is not None:
        s = np.where(valid, s, 0.0)
    return s


def rho2(inj, plan, valid, h0=None):
    """Optimal SNR^2 over the valid samples (closed form above)."""
    h0 = float(h0 if h0 is not None else (inj.h0 if inj.h0 is not None else 1.0))
    n = np.nonzero(valid)[0]
    t = plan.t_start + n * plan.dt
    Fp, Fx = geometry.antenna_tensor(t, inj.alpha, inj.delta, inj.psi, plan.det, plan.eph)
    Ap = h0 * (1.0 + inj.cosi ** 2) / 2.0
    Ax = h0 * inj.cosi
    return float(np.sum(Fp ** 2 * Ap ** 2 + Fx ** 2 * Ax ** 2) / (2.0 * plan.sigma2))


def h0_for_rho(inj, plan, valid, rho):
    """Strain amplitude giving optimal SNR rho over the valid samples."""
    return float(rho / math.sqrt(rho2(inj, plan, valid, h0=1.0)))


def inject(x, injections, plan, valid):
    """x + sum of injected signals (each scaled to its rho); returns
    (series, list of (h0, rho^2))."""
    out = np.asarray(x, np.complex128).copy()
    info = []
    for inj in injections:
        h0 = inj.h0 if inj.h0 is not None else h0_for_rho(inj, plan, valid, inj.rho)
        out += signal(inj, plan, h0=h0, valid=valid)
        info.append((h0, rho2(inj, plan, valid, h0=h0)))
    return out, info


def valid_all(plan, gaps=()):
    return resample.valid_samples(plan.n_data, 0, plan.n_data, gaps)
