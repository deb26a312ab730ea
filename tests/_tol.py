"""Error bounds for GPU parity.

The stated bound is max|y - y_ref| <= tol * max|y_ref| with tol = 1e-4 (pole radius <= 0.99)
or 2e-3 (beyond).  A cascade of random unit-peak sections can attenuate its input by many
orders of magnitude; for a few such inputs a plain sequential float32 cascade -- the accuracy
float32 arithmetic itself allows, computed by scipy.signal.sosfilt in float32, an independent
routine, on the same input, initial state and float32-rounded coefficients -- already misses
the stated bound.  For random mixes the bound is then four times that sequential error, and
never less than the stated bound.  Nothing else widens it.
"""
import numpy as np

import oracle
from workloads import designs


def fp32_sequential_error(sos, x, y_ref, zi=None):
    """Relative error of a sequential float32 cascade (scipy) against y_ref, from the same initial
    state zi ([K][2] transposed direct form II, None = zeros) as y_ref."""
    from scipy import signal
    s = np.hstack([sos[:, :3], np.ones((sos.shape[0], 1)), sos[:, 3:]]).astype(np.float32)
    x32 = np.asarray(x, np.float32)
    if zi is None:
        y = signal.sosfilt(s, x32)
    else:
        y = signal.sosfilt(s, x32, zi=np.asarray(zi, np.float32).reshape(sos.shape[0], 2))[0]
    return oracle.rel_err(y, y_ref)


def bound(sos, x=None, y_ref=None, random_mix=False, zi=None):
    tol = designs.tolerance_for(sos)
    if random_mix and x is not None and len(x):
        tol = max(tol, 4.0 * fp32_sequential_error(sos, x, y_ref, zi))
    return tol
