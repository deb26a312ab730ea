"""Pins of the float64 oracle against facts fixed by the paper and by the mathematics.

Each pin is chosen so that a plausible slip in the oracle (a swapped or
mis-signed coefficient, a dropped state term, a wrong update order, a wrong
section order) fails at least one of them; ``test_pins_catch_planted_mistakes``
plants such slips in a copy of the recurrence and checks that the pins notice.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import designs


def _resonator(r, theta, b=(1.0, 0.0, 0.0)):
    return np.array([[b[0], b[1], b[2], -2.0 * r * math.cos(theta), r * r]])


# -- pin 1: closed-form impulse response of a complex-pole biquad (Eq. 1) ------
@pytest.mark.parametrize("r,theta", [(0.9, 0.3), (0.99, 1.7), (0.5, 2.9)])
def test_impulse_response_closed_form(r, theta):
    n = 400
    k = np.arange(n)
    g = r ** k * np.sin((k + 1) * theta) / math.sin(theta)
    x = np.zeros(n)
    x[0] = 1.0
    y = oracle.sosfilt(_resonator(r, theta), x)
    np.testing.assert_allclose(y, g, rtol=0, atol=1e-12)
    # with a numerator: b0 g[n] + b1 g[n-1] + b2 g[n-2]
    b = (0.7, -1.3, 0.4)
    yb = oracle.sosfilt(_resonator(r, theta, b), x)
    gs = lambda d: np.concatenate([np.zeros(d), g[: n - d]])  # noqa: E731
    np.testing.assert_allclose(yb, b[0] * g + b[1] * gs(1) + b[2] * gs(2), rtol=0, atol=1e-12)


def test_cascade_impulse_is_convolution_of_sections():
    s1 = _resonator(0.8, 0.4, (1.0, 0.5, 0.25))
    s2 = _resonator(0.95, 2.2, (0.3, -0.2, 0.9))
    n = 300
    x = np.zeros(n)
    x[0] = 1.0
    h1 = oracle.sosfilt(s1, x)
    h2 = oracle.sosfilt(s2, x)
    h12 = np.convolve(h1, h2)[:n]
    np.testing.assert_allclose(oracle.sosfilt(np.vstack([s1, s2]), x), h12, rtol=0, atol=1e-12)
    # order of sections must not matter for the transfer function
    np.testing.assert_allclose(oracle.sosfilt(np.vstack([s2, s1]), x), h12, rtol=0, atol=1e-12)


# -- pin 2: steady-state sinusoid gain and phase -------------------------------
def test_steady_state_sinusoid():
    sos = designs.butter_lowpass(8, 0.3)
    rmax = designs.max_pole_radius(sos)
    for w in (0.1 * math.pi, 0.3 * math.pi, 0.7 * math.pi):
        h = complex(1.0)
        e1 = complex(math.cos(w), -math.sin(w))
        for b0, b1, b2, a1, a2 in sos:
            h *= (b0 + b1 * e1 + b2 * e1 * e1) / (1 + a1 * e1 + a2 * e1 * e1)
        transient = int(40 / (1 - rmax))
        n = transient + 500
        k = np.arange(n)
        y = oracle.sosfilt(sos, np.cos(w * k))
        expect = abs(h) * np.cos(w * k + math.atan2(h.imag, h.real))
        np.testing.assert_allclose(y[transient:], expect[transient:], rtol=0, atol=1e-9)


# -- pin 3: linearity, superposition, zero input --------------------------------
def test_linearity_and_zero_input():
    sos = designs.butter_lowpass(16, 0.05)
    x1 = workloads.normal_f32(11, 5000).astype(np.float64)
    x2 = workloads.normal_f32(12, 5000).astype(np.float64)
    y1, y2 = oracle.sosfilt(sos, x1), oracle.sosfilt(sos, x2)
    y12 = oracle.sosfilt(sos, 2.5 * x1 - 0.75 * x2)
    np.testing.assert_allclose(y12, 2.5 * y1 - 0.75 * y2, rtol=0, atol=1e-9 * np.abs(y12).max())
    z = oracle.sosfilt(sos, np.zeros(1000))
    assert np.all(z == 0.0)
    # zero input with a nonzero state decays as the homogeneous response and is linear in the state
    zi = np.random.default_rng(0).standard_normal((8, 2))
    h1 = oracle.sosfilt(sos, np.zeros(2000), zi=zi)
    h2 = oracle.sosfilt(sos, np.zeros(2000), zi=2 * zi)
    np.testing.assert_allclose(h2, 2 * h1, rtol=0, atol=1e-12)


# -- pin 4: chunked streaming with carried state == one shot (bit exact) --------
def test_chunked_equals_one_shot_bit_exact():
    sos = designs.random_sections(workloads.uniform_f64(5, 12).reshape(4, 3))
    x = workloads.normal_f32(3, 10007)
    y_full, zf_full = oracle.sosfilt(sos, x, return_state=True)
    cuts = [0, 1, 2, 17, 1024, 5000, 10006, 10007]
    zi = None
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        y, zi = oracle.sosfilt(sos, x[a:b], zi=zi, return_state=True)
        parts.append(y)
    assert np.array_equal(np.concatenate(parts), y_full)
    assert np.array_equal(zi, zf_full)


# -- pin 5: brute-force dense solve of the banded lower-triangular system -------
def _dense_section(row, x, z):
    """Solve A y = B x + state forcing for one section, densely (n <= 64)."""
    b0, b1, b2, a1, a2 = row
    n = len(x)
    A = np.eye(n) + a1 * np.eye(n, k=-1) + a2 * np.eye(n, k=-2)
    B = b0 * np.eye(n) + b1 * np.eye(n, k=-1) + b2 * np.eye(n, k=-2)
    rhs = B @ x
    rhs[0] += z[0]
    if n > 1:
        rhs[1] += z[1]
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_dense_solve(n):
    sos = designs.random_sections(workloads.uniform_f64(9, 9).reshape(3, 3))
    x = workloads.normal_f32(8, n).astype(np.float64)
    zi = np.random.default_rng(n).standard_normal((3, 2))
    v = x.copy()
    for k in range(3):
        v = _dense_section(sos[k], v, zi[k])
    np.testing.assert_allclose(oracle.sosfilt(sos, x, zi=zi), v, rtol=0, atol=1e-12 * max(1, np.abs(v).max()))


# -- pin 6: the permuted multi-block system of Eqs. 2-3 -------------------------
def _multiblock_matrices(N, L, c1, c2, c0=1.0):
    """Eq. 3: NL x NL block matrix on the stride-N permuted group, L x L blocks."""
    I = np.eye(L)
    R = np.eye(L, k=-1)  # lower shift: lane l feeds lane l+1
    M = np.zeros((N * L, N * L))

    def put(i, j, blk):
        M[i * L:(i + 1) * L, j * L:(j + 1) * L] += blk

    for m in range(N):
        put(m, m, c0 * I)
        if m >= 1:
            put(m, m - 1, c1 * I)
        if m >= 2:
            put(m, m - 2, c2 * I)
    put(0, N - 1, c1 * R)
    put(0, N - 2, c2 * R)
    put(1, N - 1, c2 * R)
    # columns coupling the previous group's last two samples [s[-2], s[-1]] to lane 0
    Mm = np.zeros((N * L, 2))
    Mm[0, 0] = c2
    Mm[0, 1] = c1
    Mm[L, 1] = c2
    return M, Mm


@pytest.mark.parametrize("N,L", [(2, 2), (2, 8), (4, 4), (8, 2), (8, 8), (4, 8)])
def test_permuted_multiblock_system(N, L):
    b0, b1, b2, a1, a2 = 0.8, -0.35, 0.6, -1.1, 0.45
    A, Am = _multiblock_matrices(N, L, a1, a2)
    B, Bm = _multiblock_matrices(N, L, b1, b2, b0)
    C = N * L
    rng = np.random.default_rng(N * 100 + L)
    x = rng.standard_normal(C)
    xm1 = rng.standard_normal(2)  # [x[-2], x[-1]]
    ym1 = rng.standard_normal(2)  # [y[-2], y[-1]]
    perm = np.array([l * N + m for m in range(N) for l in range(L)])  # block m = [x[m], x[m+N], ...]
    xg = x[perm]
    yg = np.linalg.solve(A, B @ xg + Bm @ xm1 - Am @ ym1)  # Eq. 2
    y = np.empty(C)
    y[perm] = yg
    # the same state in transposed direct form II
    zi = np.array([[b1 * xm1[1] + b2 * xm1[0] - a1 * ym1[1] - a2 * ym1[0], b2 * xm1[1] - a2 * ym1[1]]])
    y_or = oracle.sosfilt(np.array([[b0, b1, b2, a1, a2]]), x, zi=zi)
    np.testing.assert_allclose(y_or, y, rtol=0, atol=1e-11 * np.abs(y).max())


# -- pin 7: an independent library routine --------------------------------------
def test_matches_scipy_sosfilt():
    signal = pytest.importorskip("scipy.signal")
    sos = designs.butter_lowpass(16, 0.05)
    x = workloads.normal_f32(1, 20000)
    zi = np.random.default_rng(1).standard_normal((8, 2)) * 1e-3
    sp_sos = np.hstack([sos[:, :3], np.ones((8, 1)), sos[:, 3:]])
    y_sp, zf_sp = signal.sosfilt(sp_sos, x.astype(np.float64), zi=zi)
    y, zf = oracle.sosfilt(sos, x, zi=zi, return_state=True)
    np.testing.assert_allclose(y, y_sp, rtol=0, atol=1e-12 * np.abs(y_sp).max())
    np.testing.assert_allclose(zf, zf_sp, rtol=0, atol=1e-12 * np.abs(zf_sp).max())


def test_batch_matches_single():
    sos_list = [designs.butter_lowpass(2 * k, 0.2) for k in (1, 2, 4, 8)]
    xs = [workloads.normal_f32(50 + i, 1000 + 37 * i) for i in range(4)]
    ys, zfs = oracle.sosfilt_batch(sos_list, xs, threads=3)
    for s, x, y, zf in zip(sos_list, xs, ys, zfs):
        y1, zf1 = oracle.sosfilt(s, x, return_state=True)
        assert np.array_equal(y, y1) and np.array_equal(zf, zf1)


def test_edge_sizes():
    sos = designs.butter_lowpass(4, 0.2)
    assert oracle.sosfilt(sos, np.zeros(0, np.float32)).shape == (0,)
    y, zf = oracle.sosfilt(sos, np.ones(1, np.float32), return_state=True)
    assert y[0] == pytest.approx(sos[0, 0] * sos[1, 0])
    assert zf.shape == (2, 2)


# -- the pins catch planted mistakes (mutations of a Python copy of the recurrence)
def _mutant(kind):
    def run(sos, x, zi=None):
        sos = np.asarray(sos, dtype=np.float64).reshape(-1, 5)
        K = sos.shape[0]
        z = np.zeros((K, 2)) if zi is None else np.array(zi, dtype=np.float64).reshape(K, 2)
        out = np.empty(len(x))
        order = range(K - 1, -1, -1) if kind == "reversed_sections_with_state" else range(K)
        for i, v in enumerate(np.asarray(x, dtype=np.float64)):
            for k in order:
                b0, b1, b2, a1, a2 = sos[k]
                if kind == "swap_a":
                    a1, a2 = a2, a1
                if kind == "sign_a1":
                    a1 = -a1
                if kind == "swap_b":
                    b1, b2 = b2, b1
                y = b0 * v + z[k, 0]
                z[k, 0] = b1 * v - a1 * y + (0.0 if kind == "drop_z2" else z[k, 1])
                z[k, 1] = b2 * v - a2 * y
                v = y
            out[i] = v
        return out
    return run


@pytest.mark.parametrize("kind", ["swap_a", "sign_a1", "swap_b", "drop_z2", "reversed_sections_with_state"])
def test_pins_catch_planted_mistakes(kind):
    bad = _mutant(kind)
    good = _mutant("none")
    # the faithful copy passes the closed-form impulse pin ...
    r, th, b = 0.9, 0.3, (0.7, -1.3, 0.4)
    n = 64
    k = np.arange(n)
    g = r ** k * np.sin((k + 1) * th) / math.sin(th)
    gs = lambda d: np.concatenate([np.zeros(d), g[: n - d]])  # noqa: E731
    expect = b[0] * g + b[1] * gs(1) + b[2] * gs(2)
    x = np.zeros(n)
    x[0] = 1.0
    np.testing.assert_allclose(good(_resonator(r, th, b), x), expect, atol=1e-12)
    # ... and every mutant fails either it or the state-carrying dense pin
    caught = not np.allclose(bad(_resonator(r, th, b), x), expect, atol=1e-9)
    sos = designs.random_sections(workloads.uniform_f64(9, 9).reshape(3, 3))
    xx = workloads.normal_f32(8, 40).astype(np.float64)
    zi = np.random.default_rng(40).standard_normal((3, 2))
    v = xx.copy()
    for s in range(3):
        v = _dense_section(sos[s], v, zi[s])
    caught = caught or not np.allclose(bad(sos, xx, zi=zi), v, atol=1e-9)
    assert caught, kind


@pytest.mark.parametrize("K", [1, 2, 3, 8])
@pytest.mark.parametrize("threads", [1, 2, 5])
def test_wavefront_host_baseline_is_bit_identical(K, threads):
    # the multi-core wavefront (Sec. III-A) hands each section's state from group to group in order,
    # so it must reproduce the sequential oracle exactly, output and final state
    from workloads import designs
    sos = designs.random_sections(np.random.default_rng(K).uniform(size=(K, 3)))
    zi = np.random.default_rng(100 + K).standard_normal((K, 2)) * 0.1
    for n, block in [(0, 64), (1, 64), (63, 64), (64, 64), (5 * 64 + 3, 64), (20000, 4096)]:
        x = np.random.default_rng(n + K).standard_normal(n).astype(np.float32)
        y, zf = oracle.sosfilt(sos, x, zi=zi, return_state=True)
        y2, zf2 = oracle.sosfilt_wavefront(sos, x, zi=zi, return_state=True, threads=threads, block=block)
        assert np.array_equal(y, y2)
        assert np.array_equal(zf, zf2)
