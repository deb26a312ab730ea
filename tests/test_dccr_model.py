"""The float64 model of the kernel's algorithm agrees with the oracle and with the paper's printed algebra."""
import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

from . import dccr_model as M


def test_first_level_taps_match_eq23():
    # Eq. 23 with b0 = 1: e_B = b2 + a2 - a1 b1, f_B = a2 b2, c_B = a2 b1 - a1 b2, d_B = b1 - a1
    b1, b2, a1, a2 = 0.37, -0.81, -1.23, 0.64
    taps = M.first_level_taps(1.0, b1, b2, a1, a2)
    assert taps[0] == 1.0
    assert taps[1] == pytest.approx(b1 - a1)
    assert taps[2] == pytest.approx(b2 + a2 - a1 * b1)
    assert taps[3] == pytest.approx(a2 * b1 - a1 * b2)
    assert taps[4] == pytest.approx(a2 * b2)


def test_level_coeffs_square_the_poles():
    # each level maps the poles p to p^2 (Graeffe), so level i has poles p^(2^i)
    r, th = 0.97, 0.61
    a1, a2 = -2 * r * math.cos(th), r * r
    e, f = M.level_coeffs(a1, a2, 6)
    for i in range(7):
        p = (r * complex(math.cos(th), math.sin(th))) ** (2 ** i)
        assert e[i] == pytest.approx(-2 * p.real, abs=1e-12)
        assert f[i] == pytest.approx(abs(p) ** 2, abs=1e-12)


def test_level_polynomial_has_three_taps():
    # A(z) Q_i(z) = 1 + e_i z^-(2^i) + f_i z^-(2^(i+1)): the level-i recurrence of the reduction
    a1, a2 = -1.31, 0.72
    D = 5
    e, f = M.level_coeffs(a1, a2, D)
    Q = M.q_tables(a1, a2, D)
    for i in range(1, D + 1):
        full = M.poly_mul(Q[i], [1.0, a1, a2])
        s = 1 << i
        expect = np.zeros(2 * s + 1)
        expect[0], expect[s], expect[2 * s] = 1.0, e[i], f[i]
        np.testing.assert_allclose(full, expect, atol=1e-12)


def test_eq17_as_printed():
    """Eq. 17 fixes how the initial outputs enter the first retained odd row of each level.

    The state moved to the right-hand side forces row 0 with -(a2 y[-2] + a1 y[-1]) and row 1
    with -a2 y[-1]; after i levels row 2^i - 1 carries -(h_i y[-2] + g_i y[-1]) with
    h_0 = a2, g_0 = a1, h_{i+1} = -e_i h_i, g_{i+1} = f_i - e_i g_i.  The injection tables
    Q_i used by the kernel must give exactly these numbers.
    """
    a1, a2 = -1.31, 0.72
    D = 6
    e, f = M.level_coeffs(a1, a2, D)
    h, g = [a2], [a1]
    for i in range(D):
        h.append(-e[i] * h[i])
        g.append(f[i] - e[i] * g[i])
    Q = M.q_tables(a1, a2, D)
    for i in range(0, D + 1):
        m = (1 << i) - 1
        q = lambda k: Q[i][k] if 0 <= k < len(Q[i]) else 0.0  # noqa: E731
        assert q(m) * a2 == pytest.approx(h[i], rel=1e-12, abs=1e-300)
        assert q(m) * a1 + q(m - 1) * a2 == pytest.approx(g[i], rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("N,L", [(2, 2), (4, 2), (8, 4), (16, 8), (32, 4), (64, 2)])
def test_single_group_zero_state(N, L):
    sos = designs.random_sections(workloads.uniform_f64(N * L, 3, stream=1).reshape(1, 3))
    x = workloads.normal_f32(N + L, N * L).astype(np.float64)
    y, _, _ = M.filter_section_group_lanes(x, sos[0], N, L, np.zeros(2))
    np.testing.assert_allclose(y, oracle.sosfilt(sos, x), rtol=0, atol=1e-10 * np.abs(y).max())


@pytest.mark.parametrize("N,L", [(4, 4), (32, 8), (64, 4)])
def test_single_group_with_state(N, L):
    sos = designs.random_sections(workloads.uniform_f64(7, 3, stream=1).reshape(1, 3))
    x = workloads.normal_f32(N, N * L).astype(np.float64)
    zi = np.array([0.7, -1.9])
    y, tg, _ = M.filter_section_group_lanes(x, sos[0], N, L, zi)
    y_ref, zf_ref = oracle.sosfilt(sos, x, zi=zi[None], return_state=True)
    np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-10 * np.abs(y_ref).max())
    # group carry (Eq. 25): terminal state = zero-state carry + T^C zi
    TC = np.linalg.matrix_power(M.transition(sos[0, 3], sos[0, 4]), N * L)
    np.testing.assert_allclose(tg + TC @ zi, zf_ref[0], rtol=0, atol=1e-10 * np.abs(zf_ref).max())


@pytest.mark.parametrize("normalize", [False, True])
@pytest.mark.parametrize("K,N,L,n", [(1, 8, 4, 1000), (2, 4, 4, 33), (4, 16, 4, 64 * 5), (8, 32, 2, 777),
                                     (3, 2, 2, 9), (8, 64, 2, 128)])
def test_cascade_many_groups(K, N, L, n, normalize):
    u = workloads.uniform_f64(K * 31 + n, 3 * K, stream=1).reshape(K, 3)
    sos = designs.random_sections(u)
    x = workloads.normal_f32(K + n, n)
    zi = np.random.default_rng(n).standard_normal((K, 2)) * 0.1
    y, zf = M.sosfilt_model(sos, x, N, L, zi=zi, normalize=normalize)
    y_ref, zf_ref = oracle.sosfilt(sos, x, zi=zi, return_state=True)
    np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-9 * np.abs(y_ref).max())
    np.testing.assert_allclose(zf, zf_ref, rtol=0, atol=1e-9 * max(1.0, np.abs(zf_ref).max()))


def test_lookback_composition_matches_sequential():
    a1, a2 = -1.2, 0.5
    TC = np.linalg.matrix_power(M.transition(a1, a2), 7)
    rng = np.random.default_rng(3)
    for j in (0, 1, 5, 31, 32, 33, 70):
        locals_ = [rng.standard_normal(2) for _ in range(j)]
        glob = rng.standard_normal(2)
        # sequential: walk forward from the global carry
        z = glob.copy()
        for k in range(j - 1, -1, -1):
            z = locals_[k] + TC @ z
        np.testing.assert_allclose(M.lookback_compose(locals_, glob, TC), z, rtol=1e-12, atol=1e-12)
