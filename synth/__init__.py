"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the F-statistic method.  It only draws
random numbers and lays out plain data: the plan constants (detector site,
analytic ephemeris constants, sampling), complex Gaussian noise, gap
intervals, template grids and injection parameters.  Everything that
*computes* a time map, a beam pattern, a phase, a resampled series or 2F lives
either in the CUDA library (``paper_0912_4255_gb300``) or in the FP64 oracle
(``oracle``); the two never import each other and share only this module.

Workload sizes follow the search configurations of the barycentric-resampling
F-statistic paper (Patel, Siemens, Dupuis, Betzwieser, LIGO-P0900301):

* ``tiny``   : 12 h at dt = 0.5 s (86,400 samples), FFT 2^17, one template,
               nearest-neighbour resampling, one injection at +0.7 Hz.
* ``search`` : 10 d at dt = 0.5 s (1,728,000 samples), FFT 2^22, 10 % gaps in
               1-6 h blocks, 1024 sky points x 8 spindowns, 8-tap sinc.
* ``batch``  : 4096 templates with spans of 1-10 d, per-template gaps 0-20 %,
               FFT length next_pow2(N_b) per template.
* ``stress`` : 30 d at dt = 0.25 s (10,368,000 samples), FFT 2^24, f_h = 1 kHz,
               spindown down to -1e-8 Hz/s.
* ``diff``   : 5 d at dt = 0.5 s (864,000 samples), 10 % gaps, candidates
               near 20 injections for the gradient.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------
# plan constants (plain data)
# --------------------------------------------------------------------------

NEAREST, SINC = 0, 1
WIN_RECT, WIN_LANCZOS = 0, 1
PREC_MIXED, PREC_FP64, PREC_FP32 = 0, 1, 2

C_LIGHT = 299792458.0  # m/s, exact by definition of the metre

DEG = math.pi / 180.0


@dataclasses.dataclass
class Detector:
    """Interferometer site: geodetic latitude/longitude (east positive),
    arm-bisector azimuth gamma (counter-clockwise from local East) and the
    radius of a spherical Earth."""
    lat_rad: float = 46.45 * DEG
    lon_rad: float = -119.41 * DEG
    gamma_rad: float = 171.8 * DEG
    radius_m: float = 6371000.0


@dataclasses.dataclass
class Ephem:
    """Analytic ephemeris: circular 1 AU orbit in the ecliptic, Sun at the
    Solar System barycentre, uniform sidereal spin.  Phases are the orbital
    longitude and the Greenwich sidereal angle at t = 0."""
    au_m: float = 1.495978707e11
    year_s: float = 365.25 * 86400.0
    sidereal_day_s: float = 86164.0905
    obliquity_rad: float = 23.44 * DEG
    orb_phase0: float = 0.0
    sid_phase0: float = 0.0


@dataclasses.dataclass
class PlanDesc:
    """Everything that is fixed for a batch of templates (mirrors
    ``fstat_plan_desc`` of the C header)."""
    dt: float = 0.5
    t_start: float = 0.0
    n_data: int = 86400
    f_het: float = 100.0
    sigma2: float = 1.0
    n_fft: int = 1 << 17
    interp: int = NEAREST
    taps: int = 8
    window: int = WIN_LANCZOS
    precision: int = PREC_MIXED
    det: Detector = dataclasses.field(default_factory=Detector)
    eph: Ephem = dataclasses.field(default_factory=Ephem)
    max_templates: int = 1

    def replace(self, **kw) -> "PlanDesc":
        return dataclasses.replace(self, **kw)


# template record, one row per template (mirrors ``fstat_template``)
TEMPLATE_DTYPE = np.dtype([
    ("alpha", np.float64), ("delta", np.float64), ("fdot", np.float64),
    ("span_start", np.int64), ("span_len", np.int64),
    ("gap_off", np.int64), ("n_gaps", np.int64),
    ("n_fft", np.int64), ("out_off", np.int64),
    ("fddot", np.float64),
])


def make_templates(alpha, delta, fdot, span_start=0, span_len=None, gap_off=0,
                   n_gaps=0, n_fft=0, out_off=-1, n_data=None, fddot=0.0) -> np.ndarray:
    """Pack per-template parameters (broadcast) into a TEMPLATE_DTYPE array.

    ``n_fft = 0`` means "the plan's n_fft"; ``out_off = -1`` means
    ``index * n_fft``; ``fddot`` is the second spindown.
    """
    alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    n = alpha.size
    if span_len is None:
        if n_data is None:
            raise ValueError("span_len or n_data required")
        span_len = n_data
    t = np.zeros(n, dtype=TEMPLATE_DTYPE)
    t["alpha"] = alpha
    t["delta"] = np.broadcast_to(np.asarray(delta, np.float64), (n,))
    t["fdot"] = np.broadcast_to(np.asarray(fdot, np.float64), (n,))
    t["span_start"] = np.broadcast_to(np.asarray(span_start, np.int64), (n,))
    t["span_len"] = np.broadcast_to(np.asarray(span_len, np.int64), (n,))
    t["gap_off"] = np.broadcast_to(np.asarray(gap_off, np.int64), (n,))
    t["n_gaps"] = np.broadcast_to(np.asarray(n_gaps, np.int64), (n,))
    t["n_fft"] = np.broadcast_to(np.asarray(n_fft, np.int64), (n,))
    t["out_off"] = np.broadcast_to(np.asarray(out_off, np.int64), (n,))
    t["fddot"] = np.broadcast_to(np.asarray(fddot, np.float64), (n,))
    return t


# --------------------------------------------------------------------------
# random inputs
# --------------------------------------------------------------------------

def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def complex_noise(n: int, sigma2: float, seed: int, dtype=np.complex64) -> np.ndarray:
    """Circular complex Gaussian noise with E|n|^2 = sigma2 (Re, Im each
    N(0, sigma2/2))."""
    g = rng(seed)
    s = math.sqrt(sigma2 / 2.0)
    out = np.empty(n, dtype=dtype)
    out.real = g.standard_normal(n) * s
    out.imag = g.standard_normal(n) * s
    return out


def gap_intervals(n_data: int, frac: float, min_len: int, max_len: int,
                  seed: int, max_tries: int = 100000) -> np.ndarray:
    """Non-overlapping [start, end) sample intervals, lengths uniform in
    [min_len, max_len], drawn until at least ``frac`` of the samples are
    covered.  Returned sorted, shape (k, 2), int64.  Gaps never touch the
    first or last sample, so every span keeps data at both ends."""
    g = rng(seed)
    target = int(round(frac * n_data))
    iv: list[tuple[int, int]] = []
    covered = 0
    tries = 0
    while covered < target and tries < max_tries:
        tries += 1
        ln = int(g.integers(min_len, max_len + 1))
        ln = min(ln, target - covered) if target - covered >= min_len else ln
        if ln >= n_data - 2:
            break
        s = int(g.integers(1, n_data - ln - 1))
        e = s + ln
        # keep a margin of one sample between gaps so that they stay separate
        if any(not (e + 1 <= a or s >= b + 1) for a, b in iv):
            continue
        iv.append((s, e))
        covered += ln
    iv.sort()
    return np.asarray(iv, dtype=np.int64).reshape(-1, 2)


def zero_gaps(x: np.ndarray, gaps: np.ndarray) -> np.ndarray:
    """Set the samples inside the gap intervals to zero (no data taken)."""
    x = x.copy()
    for s, e in gaps:
        x[s:e] = 0
    return x


def fibonacci_sky(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Near-uniform sky grid (Fibonacci sphere): right ascension alpha in
    [0, 2 pi), declination delta in (-pi/2, pi/2)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    golden = math.pi * (3.0 - math.sqrt(5.0))
    alpha = np.mod(golden * i, 2.0 * math.pi)
    delta = np.arcsin(z)
    return alpha, delta


def random_sky(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    g = rng(seed)
    alpha = g.uniform(0.0, 2.0 * math.pi, n)
    delta = np.arcsin(g.uniform(-1.0, 1.0, n))
    return alpha, delta


@dataclasses.dataclass
class Injection:
    """Amplitude and Doppler parameters of one injected signal: strain
    amplitude h0 (or target SNR rho), inclination cos(iota), polarisation
    psi, initial phase phi0, sky (alpha, delta), frequency offset df above
    the heterodyne frequency, spindown fdot and second spindown fddot."""
    alpha: float
    delta: float
    df: float
    fdot: float
    psi: float
    cosi: float
    phi0: float
    rho: float = 20.0
    h0: float | None = None
    fddot: float = 0.0


def random_injection(seed: int, df: float, fdot: float = 0.0, rho: float = 20.0,
                     alpha: float | None = None, delta: float | None = None,
                     fddot: float = 0.0) -> Injection:
    g = rng(seed)
    a = g.uniform(0.0, 2.0 * math.pi) if alpha is None else alpha
    d = math.asin(g.uniform(-1.0, 1.0)) if delta is None else delta
    psi = g.uniform(0.0, math.pi)
    cosi = g.uniform(-1.0, 1.0)
    phi0 = g.uniform(0.0, 2.0 * math.pi)
    return Injection(alpha=a, delta=d, df=df, fdot=fdot, psi=psi, cosi=cosi,
                     phi0=phi0, rho=rho, fddot=fddot)


# injection record, one row per injected signal (mirrors ``fstat_injection``)
INJECTION_DTYPE = np.dtype([
    ("alpha", np.float64), ("delta", np.float64), ("psi", np.float64), ("cosi", np.float64),
    ("phi0", np.float64), ("h0", np.float64), ("df", np.float64), ("fdot", np.float64),
    ("fddot", np.float64), ("span_start", np.int64), ("span_len", np.int64),
])


def injection_records(injections, h0, span_start, span_len) -> np.ndarray:
    """Pack Injection objects with amplitudes h0 and spans (broadcast) into
    an INJECTION_DTYPE array."""
    n = len(injections)
    r = np.zeros(n, dtype=INJECTION_DTYPE)
    for name in ("alpha", "delta", "psi", "cosi", "phi0", "df", "fdot", "fddot"):
        r[name] = [getattr(i, name) for i in injections]
    r["h0"] = np.broadcast_to(np.asarray(h0, np.float64), (n,))
    r["span_start"] = np.broadcast_to(np.asarray(span_start, np.int64), (n,))
    r["span_len"] = np.broadcast_to(np.asarray(span_len, np.int64), (n,))
    return r


def random_injection_records(n: int, seed: int, df: float, h0: float, span_len: int,
                             span_start0: int = 0) -> np.ndarray:
    """n injections on consecutive spans of span_len samples: isotropic sky,
    uniform psi in [0, pi), cos(iota) in [-1, 1], phi0 in [0, 2 pi); common
    df and h0, no spindown."""
    g = rng(seed)
    r = np.zeros(n, dtype=INJECTION_DTYPE)
    r["alpha"] = g.uniform(0.0, 2.0 * math.pi, n)
    r["delta"] = np.arcsin(g.uniform(-1.0, 1.0, n))
    r["psi"] = g.uniform(0.0, math.pi, n)
    r["cosi"] = g.uniform(-1.0, 1.0, n)
    r["phi0"] = g.uniform(0.0, 2.0 * math.pi, n)
    r["h0"] = h0
    r["df"] = df
    r["span_start"] = span_start0 + np.arange(n, dtype=np.int64) * span_len
    r["span_len"] = span_len
    return r


# --------------------------------------------------------------------------
# SFT inputs (the data product of Eq. e25) for the front end
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SftDesc:
    """Front-end parameters (mirrors ``fstat_sft_desc``): raw samples per SFT
    and raw sampling interval, the stored bins k_lo .. k_lo + n_bins - 1 of
    every SFT, the heterodyne bin k_het (f_h = k_het / T_SFT), the bins per
    SFT of the output band (output interval T_SFT / band_bins), Dirichlet
    terms on each side, running-median window (0: no normalisation), Tukey
    taper fraction of the band and time-domain taper at chunk ends."""
    sft_len: int = 2048
    dt_raw: float = 1.0 / 256.0
    k_lo: int = 0
    n_bins: int = 0
    k_het: int = 0
    band_bins: int = 64
    dirichlet_terms: int = 16
    median_window: int = 0
    tukey_frac: float = 0.0
    edge_taper: int = 0

    def replace(self, **kw) -> "SftDesc":
        return dataclasses.replace(self, **kw)

    @property
    def t_sft(self) -> float:
        return self.sft_len * self.dt_raw


def sft_slots(n_slots: int, missing: int, seed: int, max_run: int = 3) -> np.ndarray:
    """Indices of the SFTs present among n_slots consecutive SFT slots, with
    ``missing`` slots removed in runs of 1..max_run (never the first)."""
    g = rng(seed)
    keep = np.ones(n_slots, bool)
    while (~keep).sum() < missing:
        a = int(g.integers(1, n_slots))
        keep[a:a + int(g.integers(1, max_run + 1))] = False
    return np.nonzero(keep)[0]


def raw_sinusoids(n: int, dt: float, freqs, amps, phases, t0: float = 0.0) -> np.ndarray:
    """Real series sum_i A_i cos(2 pi f_i (t - t0) + phi_i) at t = t0 + j dt."""
    t = np.arange(n) * dt
    x = np.zeros(n)
    for f, a, p in zip(freqs, amps, phases):
        x += a * np.cos(2.0 * math.pi * f * t + p)
    return x


def sfts_of(x_raw: np.ndarray, slots, sft_len: int, k_lo: int, n_bins: int,
            dtype=np.complex64) -> np.ndarray:
    """SFT bins k_lo .. k_lo + n_bins - 1 of the SFTs at the given slots of a
    raw real series (Eq. e25 by numpy's FFT), [len(slots), n_bins]."""
    out = np.empty((len(slots), n_bins), dtype)
    for i, a in enumerate(slots):
        X = np.fft.fft(x_raw[a * sft_len:(a + 1) * sft_len])
        out[i] = X[k_lo:k_lo + n_bins]
    return out


def sft_noise(n_sft: int, n_bins: int, sft_len: int, sigma2_raw: float, seed: int,
              dtype=np.complex64) -> np.ndarray:
    """SFT bins of white real noise of variance sigma2_raw drawn directly:
    away from DC and Nyquist they are independent circular complex Gaussians
    with E|X|^2 = sft_len * sigma2_raw."""
    g = rng(seed)
    s = math.sqrt(sft_len * sigma2_raw / 2.0)
    return (g.normal(0.0, s, (n_sft, n_bins)) + 1j * g.normal(0.0, s, (n_sft, n_bins))).astype(dtype)


def next_pow2(n: int) -> int:
    return 1 << max(0, int(n - 1).bit_length())


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

SEED_BASE = 4255


def tiny_plan(**kw) -> PlanDesc:
    """12 h, dt = 0.5 s, FFT 2^17, nearest neighbour."""
    p = PlanDesc(dt=0.5, n_data=86400, n_fft=1 << 17, interp=NEAREST, f_het=100.0)
    return p.replace(**kw) if kw else p


def search_plan(**kw) -> PlanDesc:
    """10 d, dt = 0.5 s, FFT 2^22, 8-tap Lanczos-windowed sinc."""
    p = PlanDesc(dt=0.5, n_data=1_728_000, n_fft=1 << 22, interp=SINC, taps=8,
                 window=WIN_LANCZOS, f_het=100.0, max_templates=8192)
    return p.replace(**kw) if kw else p


def batch_plan(**kw) -> PlanDesc:
    """Shared 10 d series; per-template spans of 1-10 d, FFT up to 2^21."""
    p = PlanDesc(dt=0.5, n_data=1_728_000, n_fft=1 << 21, interp=SINC, taps=8,
                 window=WIN_LANCZOS, f_het=100.0, max_templates=4096)
    return p.replace(**kw) if kw else p


def stress_plan(**kw) -> PlanDesc:
    """30 d at dt = 0.25 s, FFT 2^24, heterodyne at 1 kHz."""
    p = PlanDesc(dt=0.25, n_data=10_368_000, n_fft=1 << 24, interp=SINC, taps=8,
                 window=WIN_LANCZOS, f_het=1000.0, max_templates=8)
    return p.replace(**kw) if kw else p


def diff_plan(**kw) -> PlanDesc:
    """5 d at dt = 0.5 s, 10 % gaps, for the gradient."""
    p = PlanDesc(dt=0.5, n_data=864_000, n_fft=1 << 21, interp=SINC, taps=8,
                 window=WIN_LANCZOS, f_het=100.0, max_templates=512)
    return p.replace(**kw) if kw else p


def search_templates(n_sky: int = 1024, n_fdot: int = 8, n_data: int = 1_728_000,
                     n_gaps: int = 0) -> np.ndarray:
    """Fibonacci-sphere sky grid x fdot = linspace(-1e-9, 0, n_fdot); all
    templates span the whole series and share one gap list."""
    a, d = fibonacci_sky(n_sky)
    fd = np.linspace(-1e-9, 0.0, n_fdot)
    A = np.repeat(a, n_fdot)
    D = np.repeat(d, n_fdot)
    F = np.tile(fd, n_sky)
    return make_templates(A, D, F, 0, n_data, 0, n_gaps)


def batch_templates(n: int, n_data: int, dt: float, seed: int,
                    min_days: float = 1.0, max_days: float = 10.0,
                    max_gap_frac: float = 0.2, fdot_min: float = -1e-9):
    """Uneven spans (uniform in [min_days, max_days]), random placement,
    random sky, fdot uniform in [fdot_min, 0], and a per-template gap list
    with a gap fraction uniform in [0, max_gap_frac] (gap blocks of 1-6 h).

    Returns (templates, gaps[k, 2]) with each template's gaps at
    ``gaps[gap_off : gap_off + n_gaps]`` in absolute sample indices."""
    g = rng(seed)
    day = int(round(86400.0 / dt))
    lens = np.minimum((g.uniform(min_days, max_days, n) * day).astype(np.int64), n_data)
    starts = np.array([int(g.integers(0, n_data - L + 1)) for L in lens], dtype=np.int64)
    alpha = g.uniform(0.0, 2.0 * math.pi, n)
    delta = np.arcsin(g.uniform(-1.0, 1.0, n))
    fdot = g.uniform(fdot_min, 0.0, n)
    gap_lists = []
    offs = np.zeros(n, np.int64)
    cnts = np.zeros(n, np.int64)
    off = 0
    hour = int(round(3600.0 / dt))
    for i in range(n):
        frac = float(g.uniform(0.0, max_gap_frac))
        gi = gap_intervals(int(lens[i]), frac, hour, 6 * hour, seed=int(g.integers(1 << 31)))
        gi = gi + starts[i]
        gap_lists.append(gi)
        offs[i] = off
        cnts[i] = len(gi)
        off += len(gi)
    gaps = np.concatenate(gap_lists, axis=0) if off else np.zeros((0, 2), np.int64)
    t = make_templates(alpha, delta, fdot, starts, lens, offs, cnts)
    return t, gaps.astype(np.int64)
