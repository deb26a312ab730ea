"""Pins of the seeded input generators and the filter designs (inputs shared by both sides)."""
import cmath
import math
import os

import numpy as np
import pytest

import workloads
from workloads import designs


def _load_kat():
    """Philox4x32-10 known-answer vectors published with Random123 (Salmon et al., SC'11)."""
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v, 16) for v in line.split()]
            assert len(w) == 10, line
            rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


KAT = _load_kat()


def test_kat_fixture_complete():
    assert len(KAT) == 3


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    assert tuple(workloads.philox4x32_10_c(ctr, key)) == out
    got = workloads.philox4x32_10_np(*[np.array([c]) for c in ctr], key[0], key[1])
    assert tuple(int(v[0]) for v in got) == out


def test_c_generator_matches_numpy_restatement():
    for seed, stream, n in [(0, 0, 1), (1, 0, 1001), (1 << 40, 7, 4096)]:
        np.testing.assert_array_equal(workloads.uniform_f64(seed, n, stream), workloads.uniform_f64_np(seed, n, stream))
        a = workloads.normal_f32(seed, n, stream)
        b = workloads.normal_f32_np(seed, n, stream)
        # same uniforms; libm vs numpy transcendental rounding may differ in the last double ulp
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)


def test_normal_moments_and_threading_invariance():
    x = workloads.normal_f32(0, 1 << 20)
    assert abs(float(x.mean())) < 5e-3 and abs(float(x.std()) - 1.0) < 5e-3
    # prefixes are stable: the sample at index i does not depend on n or on the thread split
    y = workloads.normal_f32(0, 1000)
    np.testing.assert_array_equal(x[:1000], y)


def test_sinusoid_added():
    n = 4096
    a = workloads.normal_f32(4, n)
    b = workloads.normal_f32(4, n, sin_amp=1.0, sin_omega=0.32 * math.pi)
    k = np.arange(n)
    np.testing.assert_allclose(b.astype(np.float64) - a, np.sin(0.32 * math.pi * k), atol=1e-6)


def _h(sos, w):
    e1 = cmath.exp(-1j * w)
    h = 1.0
    for b0, b1, b2, a1, a2 in sos:
        h *= (b0 + b1 * e1 + b2 * e1 * e1) / (1 + a1 * e1 + a2 * e1 * e1)
    return h


def test_butterworth_order2_closed_form():
    # K = tan(wc/2), D = 1 + sqrt(2) K + K^2 : b = K^2/D [1,2,1], a1 = 2(K^2-1)/D, a2 = (1 - sqrt(2) K + K^2)/D
    sos = designs.butter_lowpass(2, 0.2)
    assert sos.shape == (1, 5)
    assert sos[0, 0] == pytest.approx(0.0674552738890719, abs=1e-15)
    assert sos[0, 3] == pytest.approx(-1.1429805025399011, abs=1e-15)
    assert sos[0, 4] == pytest.approx(0.4128015980961886, abs=1e-15)
    assert list(sos[0, :3] / sos[0, 0]) == pytest.approx([1, 2, 1])


@pytest.mark.parametrize("order,wn", [(2, 0.2), (4, 0.2), (8, 0.1), (16, 0.05), (16, 0.2)])
def test_butterworth_response(order, wn):
    sos = designs.butter_lowpass(order, wn)
    assert sos.shape == (order // 2, 5)
    assert abs(_h(sos, 0.0)) == pytest.approx(1.0, abs=1e-9)
    assert abs(_h(sos, math.pi * wn)) == pytest.approx(1 / math.sqrt(2), abs=1e-9)
    # |H|^2 = 1 / (1 + (tan(w/2)/tan(wc/2))^(2 order)) on the bilinear-warped axis
    for w in np.linspace(0.01, 3.1, 13):
        ratio = math.tan(w / 2) / math.tan(math.pi * wn / 2)
        assert abs(_h(sos, w)) ** 2 == pytest.approx(1 / (1 + ratio ** (2 * order)), rel=1e-7, abs=1e-14)
    radii = [abs(np.roots([1, a1, a2])).max() for _, _, _, a1, a2 in sos]
    assert radii == sorted(radii)
    signal = pytest.importorskip("scipy.signal")
    ref = signal.butter(order, wn, output="sos")
    for w in np.linspace(0.0, 3.0, 7):
        _, hr = signal.sosfreqz(ref, worN=[w])
        assert abs(_h(sos, w)) == pytest.approx(abs(hr[0]), rel=1e-7, abs=1e-12)


def test_order16_design_pole_radii():
    sos = designs.butter_lowpass(16, 0.05)
    assert 0.98 < designs.max_pole_radius(sos) < 0.99
    assert designs.tolerance_for(sos) == 1e-4


def test_resonator_bank():
    sos = designs.resonator_bank()
    assert sos.shape == (8, 5)
    assert designs.max_pole_radius(sos) == pytest.approx(0.999, abs=1e-12)
    assert designs.tolerance_for(sos) == 2e-3
    for k in range(8):
        th = math.pi * (0.30 + 0.04 * k / 7)
        assert abs(_h(sos[k:k + 1], th)) == pytest.approx(1.0, abs=1e-12)
        assert abs(_h(sos[k:k + 1], 0.0)) < 1e-12 and abs(_h(sos[k:k + 1], math.pi)) < 1e-12


def test_random_sections():
    u = workloads.uniform_f64(1000, 8 * 3, stream=1).reshape(8, 3)
    sos = designs.random_sections(u)
    for row in sos:
        r = abs(np.roots([1, row[3], row[4]])).max()
        assert 0.6 <= r <= 0.995
        assert row[0] == pytest.approx(row[2])
        w = np.linspace(0, math.pi, 4001)
        peak = max(abs(_h(row[None], wi)) for wi in w)
        assert peak <= 1.0 + 1e-3


def test_batched_mix_recipe():
    orders, lens = [], []
    for i in range(400):
        sos, n, seed = workloads.batched_signal(i)
        K = sos.shape[0]
        orders.append(2 * K)
        lens.append(n)
        assert seed == 1000 + i
        assert 2 ** 10 - 1 <= n <= 2 ** 22 + 1
        assert designs.max_pole_radius(sos) < 0.9951
    assert set(orders) == {2, 4, 8, 16}
    # log-uniform lengths: the median of log2 length near 16
    assert 15.0 < np.median(np.log2(lens)) < 17.0
    # deterministic
    a, b = workloads.batched_signal(7), workloads.batched_signal(7)
    assert a[1] == b[1] and np.array_equal(a[0], b[0])


def test_serving_mix_recipe():
    from collections import Counter
    cnt = Counter(2 * workloads.serving_stream(s).shape[0] for s in range(2000))
    for order, share in zip(workloads.SERVE_ORDERS, workloads.SERVE_ORDER_SHARES):
        assert abs(cnt[order] / 2000 - share) < 0.04
    lens = [workloads.serving_chunk_len(s, c) for s in range(50) for c in range(20)]
    assert min(lens) >= 4096 and max(lens) <= 65536
    assert abs(np.mean(lens) - (4096 + 65536) / 2) < 2500
    assert np.array_equal(workloads.serving_chunk(3, 5, 100), workloads.serving_chunk(3, 5, 100))
    assert not np.array_equal(workloads.serving_chunk(3, 5, 100), workloads.serving_chunk(3, 6, 100))
