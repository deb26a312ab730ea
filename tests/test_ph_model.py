"""The float64 model of the PH-factorization kernel's decomposition agrees with the oracle.

This pins the algebra of the PH kernel (lane particular solutions, the cascade lane scan through
the coupling blocks of M_N, tile folding, one homogeneous correction, the final state) on the CPU,
independently of the CUDA code.
"""
import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

from . import ph_model as PM


@pytest.mark.parametrize("K,n,W", [(1, 3 * 1024 + 5, 8), (2, 1, 8), (3, 9000, 2), (8, 40000, 8),
                                   (8, 8 * 1024 * 3 + 1, 8), (5, 2047, 4)])
def test_ph_model_matches_oracle(K, n, W):
    sos = designs.butter_lowpass(2 * K, 0.05) if K > 1 else designs.butter_lowpass(2, 0.2)
    x = workloads.normal_f32(1, n)
    zi = np.random.default_rng(K).standard_normal((K, 2)) * 0.1
    y, zf = PM.ph_filter(sos, x, zi=zi, W=W)
    y_ref, zf_ref = oracle.sosfilt(sos, x, zi=zi, return_state=True)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    assert np.abs(zf - zf_ref.reshape(-1)).max() <= 1e-12 * max(1.0, np.abs(zf_ref).max())


def test_ph_model_random_sections_and_resonators():
    for sos in (designs.random_sections(workloads.uniform_f64(7, 12).reshape(4, 3)), designs.resonator_bank()):
        x = workloads.normal_f32(3, 5000)
        y, _ = PM.ph_filter(sos, x)
        y_ref = oracle.sosfilt(sos, x)
        assert np.abs(y - y_ref).max() <= 1e-9 * np.abs(y_ref).max()


def test_coupling_blocks_are_lower_triangular():
    # the cascade transition is block lower-triangular: a section's state never feeds an earlier one
    sos = designs.butter_lowpass(8, 0.1)
    M1, _ = PM.tables([tuple(r) for r in sos], 32)
    K = sos.shape[0]
    for k in range(K):
        for j in range(k + 1, K):
            assert np.all(M1[2 * k:2 * k + 2, 2 * j:2 * j + 2] == 0.0)


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("unit_b0", [True, False])
def test_skewed_df2_particular_matches_transposed_form(K, unit_b0):
    # the skewed-pass kernel's particular solution (direct form II, sections skewed by one sample,
    # terminal state converted to transposed direct form II) equals the section-by-section
    # transposed-form particular solution, outputs and states, at the end and after any sample
    rows = workloads.uniform_f64(20 + K, 5 * K).reshape(K, 5)
    sos = designs.random_sections(rows[:, :3])
    if not unit_b0:
        sos[:, :3] *= 0.5 + rows[:, 3:4]
    coef = [tuple(r) for r in sos]
    if unit_b0:
        coef = [(1.0, b1 / b0, b2 / b0, a1, a2) for (b0, b1, b2, a1, a2) in coef]
    xb = workloads.normal_f32(40 + K, 6 * 64).reshape(6, 64)
    w_ref, states = PM.particular(coef, xb)
    for m_cap in (0, 1, 17, 63):
        w, t, cap = PM.particular_skewed_df2(coef, xb, m_cap=m_cap)
        scale = max(1.0, np.abs(states).max())
        assert np.abs(w - w_ref).max() <= 1e-11 * np.abs(w_ref).max()
        assert np.abs(t - states[:, -1]).max() <= 1e-11 * scale
        assert np.abs(cap - states[:, m_cap]).max() <= 1e-11 * scale


@pytest.mark.parametrize("n_tiles", [1, 2, 31, 32, 33, 64, 65, 97])
def test_anchored_lookback_composition_matches_oracle(n_tiles):
    # the PH kernels' fixed lookback composition (resolved carry of the last tile at a multiple of
    # 32 plus the local carries after it) reproduces the sequential carry: small groups (N = 4,
    # L = 4, W = 2) so that many tiles, across several anchors, stay cheap
    sos = designs.butter_lowpass(6, 0.1)
    n = n_tiles * 4 * 4 * 2 - 3
    x = workloads.normal_f32(90 + n_tiles, n)
    zi = np.random.default_rng(n_tiles).standard_normal((3, 2)) * 0.1
    y, zf = PM.ph_filter(sos, x, zi=zi, N=4, L=4, W=2, anchored=True)
    y_seq, zf_seq = PM.ph_filter(sos, x, zi=zi, N=4, L=4, W=2)
    y_ref, zf_ref = oracle.sosfilt(sos, x, zi=zi, return_state=True)
    assert np.abs(y - y_ref).max() <= 1e-11 * np.abs(y_ref).max()
    assert np.abs(zf - zf_ref.reshape(-1)).max() <= 1e-11 * max(1.0, np.abs(zf_ref).max())
    assert np.abs(y - y_seq).max() <= 1e-12 * np.abs(y_ref).max()
