"""Detector motion, Roemer delay and beam patterns (FP64, test oracle).

Section II of the paper: the phase of the signal (Eq. 4) contains the term
n0 . r_d(t) / c, the Roemer delay t_m (Eq. 4pt2); its time derivative is the
Doppler factor n0 . v_d / c (Eq. 11c).  The detector response is
F_+ = a cos 2psi + b sin 2psi, F_x = b cos 2psi - a sin 2psi for arms at
90 degrees (Eqs. 2-3); the paper does not print a(t), b(t) and defers to
Jaranowski, Krolak & Schutz (1998).  Two independent forms are given here:
the JKS closed form (used by the resampling path) and the contraction of the
detector tensor with the wave polarisation tensors (used for injections and
to pin the closed form).

The ephemeris is analytic: a circular orbit of radius ``au_m`` in the
ecliptic, the Sun at the barycentre, a spherical Earth spinning at the
sidereal rate, equatorial coordinates obtained by a rotation through the
obliquity.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0


def sky_vector(alpha, delta):
    """Unit vector n0(alpha, delta) towards the source, equatorial frame."""
    ca, sa = np.cos(alpha), np.sin(alpha)
    cd, sd = np.cos(delta), np.sin(delta)
    return np.stack(np.broadcast_arrays(cd * ca, cd * sa, sd), axis=-1)


def orbital_angle(t, eph):
    return eph.orb_phase0 + 2.0 * np.pi * np.asarray(t, dtype=np.float64) / eph.year_s


def sidereal_angle(t, eph, det):
    """Local sidereal angle of the detector meridian."""
    return (eph.sid_phase0 + det.lon_rad
            + 2.0 * np.pi * np.asarray(t, dtype=np.float64) / eph.sidereal_day_s)


def detector_position(t, det, eph):
    """r_d(t) in metres, SSB-centred equatorial frame: orbit + rotation."""
    phi = orbital_angle(t, eph)
    th = sidereal_angle(t, eph, det)
    ce, se = np.cos(eph.obliquity_rad), np.sin(eph.obliquity_rad)
    orb = eph.au_m * np.stack([np.cos(phi), np.sin(phi) * ce, np.sin(phi) * se], axis=-1)
    cl, sl = np.cos(det.lat_rad), np.sin(det.lat_rad)
    rot = det.radius_m * np.stack([cl * np.cos(th), cl * np.sin(th),
                                   sl * np.ones_like(th)], axis=-1)
    return orb + rot


def detector_velocity(t, det, eph):
    """v_d(t) = d r_d / dt in m/s."""
    phi = orbital_angle(t, eph)
    th = sidereal_angle(t, eph, det)
    wo = 2.0 * np.pi / eph.year_s
    ws = 2.0 * np.pi / eph.sidereal_day_s
    ce, se = np.cos(eph.obliquity_rad), np.sin(eph.obliquity_rad)
    orb = eph.au_m * wo * np.stack([-np.sin(phi), np.cos(phi) * ce, np.cos(phi) * se], axis=-1)
    cl = np.cos(det.lat_rad)
    rot = det.radius_m * ws * np.stack([-cl * np.sin(th), cl * np.cos(th),
                                        np.zeros_like(th)], axis=-1)
    return orb + rot


def roemer_delay(t, alpha, delta, det, eph):
    """t_m(t) = n0 . r_d(t) / c  (Eq. 4pt2), seconds."""
    n = sky_vector(alpha, delta)
    return detector_position(t, det, eph) @ n / C_LIGHT


def roemer_rate(t, alpha, delta, det, eph):
    """dt_m/dt = n0 . v_d(t) / c  (Eq. 11c), dimensionless Doppler factor."""
    n = sky_vector(alpha, delta)
    return detector_velocity(t, det, eph) @ n / C_LIGHT


# --------------------------------------------------------------------------
# beam patterns
# --------------------------------------------------------------------------

def beam_ab(t, alpha, delta, det, eph):
    """a(t), b(t): amplitude modulation functions of an interferometer with
    arms at 90 degrees (JKS 1998 closed form), as functions of the detector
    latitude lambda, the arm-bisector azimuth gamma (counter-clockwise from
    East), the source declination delta and the hour angle
    H = theta(t) - alpha, theta the local sidereal angle.  These are the a, b
    of Eqs. 2-3."""
    lam, gam = det.lat_rad, det.gamma_rad
    x = alpha - sidereal_angle(t, eph, det)           # alpha - phi_r - Omega_r t
    s2g, c2g = np.sin(2 * gam), np.cos(2 * gam)
    sl, cl = np.sin(lam), np.cos(lam)
    c2l, s2l = np.cos(2 * lam), np.sin(2 * lam)
    sd, cd = np.sin(delta), np.cos(delta)
    c2d, s2d = np.cos(2 * delta), np.sin(2 * delta)
    a = (s2g * (3 - c2l) * (3 - c2d) * np.cos(2 * x) / 16.0
         - c2g * sl * (3 - c2d) * np.sin(2 * x) / 4.0
         + s2g * s2l * s2d * np.cos(x) / 4.0
         - c2g * cl * s2d * np.sin(x) / 2.0
         + 0.75 * s2g * cl * cl * cd * cd)
    b = (c2g * sl * sd * np.cos(2 * x)
         + s2g * (3 - c2l) * sd * np.sin(2 * x) / 4.0
         + c2g * cl * cd * np.cos(x)
         + s2g * s2l * cd * np.sin(x) / 2.0)
    return a, b


def detector_tensor(t, det, eph):
    """d = (u u^T - v v^T)/2 for unit arm vectors u, v at azimuths
    gamma -+ 45 degrees (counter-clockwise from local East), equatorial frame.
    Shape (..., 3, 3)."""
    th = sidereal_angle(t, eph, det)
    lam = det.lat_rad
    st, ct = np.sin(th), np.cos(th)
    sl, cl = np.sin(lam), np.cos(lam)
    z = np.zeros_like(th)
    east = np.stack([-st, ct, z], axis=-1)
    north = np.stack([-sl * ct, -sl * st, cl * np.ones_like(th)], axis=-1)
    g1 = det.gamma_rad - np.pi / 4
    g2 = det.gamma_rad + np.pi / 4
    u = np.cos(g1) * east + np.sin(g1) * north
    v = np.cos(g2) * east + np.sin(g2) * north
    return 0.5 * (u[..., :, None] * u[..., None, :] - v[..., :, None] * v[..., None, :])


def polarisation_tensors(alpha, delta, psi=0.0):
    """eps_+ and eps_x for a wave from direction n0(alpha, delta), in the
    basis (e_alpha, -e_delta) rotated by the polarisation angle psi.  The
    orientation of the basis (the sign of eps_x) and the sense of psi are
    the ones of Eqs. 2-3: with them d : eps_+ = a cos 2psi + b sin 2psi and
    d : eps_x = b cos 2psi - a sin 2psi for the JKS a, b."""
    ea = np.array([-np.sin(alpha), np.cos(alpha), 0.0])
    ed = np.array([-np.sin(delta) * np.cos(alpha), -np.sin(delta) * np.sin(alpha), np.cos(delta)])
    ep = np.outer(ea, ea) - np.outer(ed, ed)
    ex = -(np.outer(ea, ed) + np.outer(ed, ea))
    c, s = np.cos(2 * psi), np.sin(2 * psi)
    return c * ep + s * ex, -s * ep + c * ex


def antenna_tensor(t, alpha, delta, psi, det, eph):
    """F_+(t), F_x(t) = d : eps_+(psi), d : eps_x(psi) (tensor contraction)."""
    d = detector_tensor(t, det, eph)
    ep, ex = polarisation_tensors(alpha, delta, psi)
    return np.einsum("...ij,ij->...", d, ep), np.einsum("...ij,ij->...", d, ex)
