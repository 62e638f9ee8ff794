"""The time map's knot spacing (no GPU): the library joins FP64 knots of
t_m(t), a(t), b(t) by cubic Hermite pieces (values and derivatives at both
ends) and, for the searches here (f_het dt <= 50, dt <= 0.5 s), puts a knot
every 2^11 grid points, 1024 s.  Checked here against the oracle's exact
functions over 10 d at several sky positions, with a Hermite interpolant
written out from its definition: the a, b error stays below 2e-6 (relative
to their range) and the delay error below 1e-8 s, which moves the phase at
f_h = 100 Hz by under 1e-6 cycles.  Doubling the piece length raises the
error about 16-fold (the h^4 law), which is what bounds the spacing."""
import numpy as np

import synth
from oracle import geometry as G
from paper_0912_4255_gb300 import autotune as at


def _hermite_max_error(f, df, t0, t1, h):
    """Largest |f - H| over [t0, t1] for the cubic Hermite pieces of f with
    knots every h seconds (evaluated at 16 points per piece)."""
    knots = np.arange(t0, t1 + h, h)
    fk, dk = f(knots), df(knots)
    worst = 0.0
    u = np.linspace(0.0, 1.0, 17)[1:-1]
    h00, h10 = 2 * u ** 3 - 3 * u ** 2 + 1, u ** 3 - 2 * u ** 2 + u
    h01, h11 = -2 * u ** 3 + 3 * u ** 2, u ** 3 - u ** 2
    for i in range(len(knots) - 1):
        t = knots[i] + u * h
        interp = h00 * fk[i] + h10 * h * dk[i] + h01 * fk[i + 1] + h11 * h * dk[i + 1]
        worst = max(worst, float(np.max(np.abs(interp - f(t)))))
    return worst


def test_default_spacing_of_the_searches():
    assert at.default_knot_log2(100.0, 0.5) == 11
    assert at.default_knot_log2(150.0, 0.5) == 10
    assert at.default_knot_log2(1000.0, 0.25) == 9
    assert at.default_knot_log2(20.0, 1.0) == 10          # longer pieces only up to dt = 0.5 s


def test_hermite_pieces_at_1024_s_meet_the_error_budget():
    d = synth.search_plan()
    det, eph = d.det, d.eph
    T = 10 * 86400.0
    eps_t = 0.5                                            # seconds for the numerical derivative of a, b
    for alpha, delta in [(0.3, 1.2), (2.0, 0.0), (4.5, -0.8), (1.0, -1.5)]:
        tm = lambda t: G.roemer_delay(t, alpha, delta, det, eph)
        dtm = lambda t: G.roemer_rate(t, alpha, delta, det, eph)
        err_t = _hermite_max_error(tm, dtm, 0.0, T, 1024.0)
        assert err_t < 1e-8, (alpha, delta, err_t)        # s; phase error at 100 Hz < 1e-6 cycles
        for k in (0, 1):
            f = lambda t, k=k: G.beam_ab(t, alpha, delta, det, eph)[k]
            df = lambda t, k=k: (f(t + eps_t) - f(t - eps_t)) / (2 * eps_t)
            err = _hermite_max_error(f, df, 0.0, 2 * 86400.0, 1024.0)
            assert err < 2e-6, (alpha, delta, k, err)
            err2 = _hermite_max_error(f, df, 0.0, 2 * 86400.0, 2048.0)
            assert 8.0 < err2 / err < 24.0                 # the h^4 law
