"""Filter designs used as synthetic workloads (inputs, not the filtering method).

Every design returns a float64 array ``sos`` of shape (K, 5) holding
``b0, b1, b2, a1, a2`` per section with ``a0 = 1`` (the biquad of Eq. 1, with
its gain kept per section).

* ``butter_lowpass(order, wn)`` -- the paper's benchmark family (Sec. IV-F):
  Butterworth low-pass of even order 2K, cutoff ``wn`` as a fraction of the
  Nyquist frequency, through the bilinear transform with pre-warping.  The
  2K analog poles ``Omega_c * exp(j*pi*(2k + 2K + 1) / (4K))`` map to
  ``z = (2 + p) / (2 - p)``; all zeros sit at z = -1.  Conjugate pole pairs
  become sections ordered by ascending pole radius, each scaled to unit gain
  at DC: ``b = (1 + a1 + a2) / 4 * [1, 2, 1]``.
* ``resonator_bank(...)`` -- the precision-stress design: eight sections with
  poles at radius 0.999 and angles evenly spaced in [0.30 pi, 0.34 pi], zeros
  at z = +1 and z = -1 (``b ~ [1, 0, -1]``), each with unit gain at its own
  pole angle.
* ``random_sections(...)`` -- stable random sections for the batched and
  serving mixes: pole radius U[0.6, 0.995], pole angle U[0.05 pi, 0.95 pi],
  a zero pair on the unit circle at angle U[0, pi], unit peak gain (maximum
  of |H| over a 16384-point grid on [0, pi] plus the pole angle).
"""
from __future__ import annotations

import math

import numpy as np


def _section_from_pole(pole: complex) -> tuple[float, float]:
    return -2.0 * pole.real, abs(pole) ** 2


def butter_lowpass(order: int, wn: float) -> np.ndarray:
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    if not 0.0 < wn < 1.0:
        raise ValueError("wn must lie in (0, 1)")
    k_sec = order // 2
    omega_c = 2.0 * math.tan(math.pi * wn / 2.0)  # pre-warped analog cutoff, T = 1
    poles = []
    for k in range(order):
        p = omega_c * complex(math.cos(math.pi * (2 * k + order + 1) / (2 * order)),
                              math.sin(math.pi * (2 * k + order + 1) / (2 * order)))
        z = (2.0 + p) / (2.0 - p)
        if z.imag > 0:  # one pole of each conjugate pair
            poles.append(z)
    assert len(poles) == k_sec, "even-order Butterworth has no real poles"
    poles.sort(key=abs)
    sos = np.zeros((k_sec, 5))
    for i, z in enumerate(poles):
        a1, a2 = _section_from_pole(z)
        g = (1.0 + a1 + a2) / 4.0
        sos[i] = [g, 2.0 * g, g, a1, a2]
    return sos


def _gain(sos_row, w: float) -> float:
    b0, b1, b2, a1, a2 = sos_row
    e1 = complex(math.cos(w), -math.sin(w))
    e2 = e1 * e1
    return abs((b0 + b1 * e1 + b2 * e2) / (1.0 + a1 * e1 + a2 * e2))


def resonator_bank(n_sections: int = 8, radius: float = 0.999, theta_lo: float = 0.30,
                   theta_hi: float = 0.34) -> np.ndarray:
    sos = np.zeros((n_sections, 5))
    for k in range(n_sections):
        frac = k / (n_sections - 1) if n_sections > 1 else 0.0
        theta = math.pi * (theta_lo + (theta_hi - theta_lo) * frac)
        a1, a2 = -2.0 * radius * math.cos(theta), radius * radius
        row = np.array([1.0, 0.0, -1.0, a1, a2])
        g = _gain(row, theta)
        row[:3] /= g
        sos[k] = row
    return sos


_GRID = np.linspace(0.0, math.pi, 16384)


def _peak_gain(row) -> float:
    b0, b1, b2, a1, a2 = row
    e1 = np.exp(-1j * _GRID)
    e2 = e1 * e1
    h = np.abs((b0 + b1 * e1 + b2 * e2) / (1.0 + a1 * e1 + a2 * e2))
    return float(h.max())


def random_sections(u: np.ndarray) -> np.ndarray:
    """Sections from uniforms ``u`` of shape (K, 3) = (radius, angle, zero angle) draws."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    sos = np.zeros((u.shape[0], 5))
    for k, (ur, ut, uz) in enumerate(u):
        r = 0.6 + (0.995 - 0.6) * ur
        theta = math.pi * (0.05 + 0.90 * ut)
        phi = math.pi * uz
        a1, a2 = -2.0 * r * math.cos(theta), r * r
        row = np.array([1.0, -2.0 * math.cos(phi), 1.0, a1, a2])
        peak = max(_peak_gain(row), _gain(row, theta))
        row[:3] /= peak
        sos[k] = row
    return sos


def max_pole_radius(sos: np.ndarray) -> float:
    r = 0.0
    for _, _, _, a1, a2 in np.asarray(sos).reshape(-1, 5):
        roots = np.roots([1.0, a1, a2])
        r = max(r, float(np.max(np.abs(roots))))
    return r


def tolerance_for(sos: np.ndarray) -> float:
    """Error bound on max|y - y_ref| / max|y_ref|: 1e-4 up to pole radius 0.99, else 2e-3."""
    return 1e-4 if max_pole_radius(sos) <= 0.99 + 1e-12 else 2e-3
