"""FP64 CPU oracle of the barycentric-resampling F-statistic.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never imports it, and it never imports the CUDA library: the two
share no code, only the seeded inputs of ``synth``.

Everything here is plain NumPy in float64 / complex128, written step by step
from the paper (Patel, Siemens, Dupuis, Betzwieser, "Implementation of
barycentric resampling for continuous wave searches in gravitational wave
data", LIGO-P0900301):

* ``geometry``  Roemer delay t_m = n.r_d/c (Eq. 4pt2), its rate (Eq. 11c),
                beam-pattern functions a(t), b(t) of Eqs. 2-3 (closed form and
                detector-tensor form).
* ``timemap``   barycentric grid t_b^k and its inverse T^k (Eqs. 11, 21).
* ``resample``  interpolation z(T^k) from z(t^k) and the gap mask (Sec. III.A.2
                steps 3-4, Sec. III.B "Gaps in the data").
* ``fstat``     the resampling F-statistic (Eqs. 19-20, 6) over all FFT bins,
                direct demodulation (Eqs. 7-8) at arbitrary frequencies, the
                single-bin form and its finite-difference gradient.
* ``inject``    signal injection (Eqs. 1-4) and the optimal SNR rho^2.
* ``candidates`` per-band top-k of 2F rows (the plain definition).
* ``frontend``  the SFT front end of Sec. III.B (normalisation, Dirichlet
                merge of Eq. e9, band selection, inverse transform, stitching).
* ``demod``     the SFT-domain demodulation F-statistic of the speed
                comparison (Sec. IV.A), from Eq. 7 and Eq. e9's kernel.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test except where the docstring says
"parity unpinned".
"""
from . import geometry, timemap, resample, fstat, inject  # noqa: F401
