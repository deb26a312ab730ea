"""Error bounds for GPU parity.

The stated bound is max|y - y_ref| <= tol * max|y_ref| with tol = 1e-4 (pole radius <= 0.99)
or 2e-3 (beyond).  A cascade of random unit-peak sections can attenuate its input by many
orders of magnitude, and then no float32 evaluation meets that bound: the rounding of the
early sections (relative to their own, much larger, outputs) reaches the output through the
later sections.  For such inputs the bound is widened to four times the error of a plain
sequential float32 cascade (scipy.signal.sosfilt in float32, an independent routine) on the
same input and coefficients -- the accuracy float32 arithmetic itself allows -- and at least four
float32 roundings of the largest intermediate (section output) signal relative to the output peak:
the parallel algorithm's corrections and carried states are of the size of the intermediate
signals, so their rounding reaches the attenuated output at that relative size.
"""
import numpy as np

import oracle
from workloads import designs


def fp32_sequential_error(sos, x, y_ref):
    from scipy import signal
    s = np.hstack([sos[:, :3], np.ones((sos.shape[0], 1)), sos[:, 3:]]).astype(np.float32)
    return oracle.rel_err(signal.sosfilt(s, np.asarray(x, np.float32)), y_ref)


EPS32 = float(np.finfo(np.float32).eps)


def intermediate_ratio(sos, x, y_ref):
    """Largest peak of the sections' outputs (float64 oracle) over the peak of the cascade output.

    Any float32 evaluation rounds the intermediate signals at a few units of EPS32 of their own
    size, and an attenuating cascade carries that absolute error to its small output.
    """
    peak_out = max(1e-300, float(np.max(np.abs(y_ref))))
    v, peak = np.asarray(x, np.float64), 0.0
    for k in range(sos.shape[0]):
        v = oracle.sosfilt(sos[k:k + 1], v)
        peak = max(peak, float(np.max(np.abs(v))))
    return peak / peak_out


def bound(sos, x=None, y_ref=None, random_mix=False):
    tol = designs.tolerance_for(sos)
    if random_mix and x is not None and len(x):
        tol = max(tol, 4.0 * fp32_sequential_error(sos, x, y_ref), 4.0 * EPS32 * intermediate_ratio(sos, x, y_ref))
    return tol
