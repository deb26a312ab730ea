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
def test_skewed_df1_particular_matches_transposed_form(K, unit_b0):
    # the skewed-pass kernel's particular solution (direct-form-I order across the cascade,
    # sections skewed by one sample, terminal state formed in transposed direct form II) equals the
    # section-by-section transposed-form particular solution, outputs and states, at the end and
    # after any sample
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
        w, t, cap = PM.particular_skewed_df1(coef, xb, m_cap=m_cap)
        scale = max(1.0, np.abs(states).max())
        assert np.abs(w - w_ref).max() <= 1e-11 * np.abs(w_ref).max()
        assert np.abs(t - states[:, -1]).max() <= 1e-11 * scale
        assert np.abs(cap - states[:, m_cap]).max() <= 1e-11 * scale


def _df2_particular_f32(coef, xb):
    """Float32 direct-form-II particular pass (u = x - a1 u[-1] - a2 u[-2], y = b0 u + b1 u[-1] +
    b2 u[-2], one rounding per multiply-add): the realisation the direct-form-I order replaced."""
    f = np.float32
    w = xb.astype(f)
    for b0, b1, b2, a1, a2 in coef:
        u1 = np.zeros(w.shape[0], f)
        u2 = np.zeros(w.shape[0], f)
        out = np.empty_like(w)
        for m in range(w.shape[1]):
            u = (np.float64(-a1) * u1 + (np.float64(-a2) * u2 + w[:, m])).astype(f)
            out[:, m] = (np.float64(f(b1)) * u1 + (np.float64(f(b2)) * u2 + np.float64(f(b0)) * u)).astype(f)
            u2, u1 = u1, u
        w = out
    return w


def test_particular_pass_float32_error_tracks_sequential_float32():
    # A high-Q cascade from the batched mix (8 random sections, pole radii up to 0.99, output peak
    # about 1e-6 of the largest section output).  Every lane block starts from zero state, so the
    # particular outputs carry the start-up transients of the inner sections; the exact correction
    # (float64 here) removes them, and what is left is the particular pass's own float32 rounding.
    # In the kernel's direct-form-I order it stays within 1.5x of a sequential float32 cascade's
    # error; the direct-form-II order, whose internal signal 1/A(z) x grows near the poles, errs
    # about 4x more on this input.
    sos, n, seed = workloads.batched_signal(28)
    x = workloads.normal_f32(seed, n)
    y_ref = oracle.sosfilt(sos, x)
    N = 64
    nl = -(-n // N)
    xb = np.zeros(nl * N, np.float32)
    xb[:n] = x
    xb = xb.reshape(nl, N)
    g = float(np.prod(sos[:, 0]))
    coef = [(1.0, b1 / b0, b2 / b0, a1, a2) for (b0, b1, b2, a1, a2) in sos]
    # the correction: each lane block's true incoming state (float64 oracle), in the b0-normalized
    # domain (section k's state scaled by the product of the later sections' b0), through the basis
    M1, H = PM.tables(coef, N)
    K = sos.shape[0]
    zscale = np.repeat([np.prod(sos[k + 1:, 0]) for k in range(K)], 2)
    zs = np.zeros((nl, 2 * K))
    z = np.zeros((K, 2))
    for blk in range(nl):
        zs[blk] = z.reshape(-1) * zscale
        _, z = oracle.sosfilt(sos, x[blk * N:(blk + 1) * N], zi=z, return_state=True)
    corr = zs @ H
    xg = (xb.astype(np.float64) * np.float32(g)).astype(np.float32)
    w1, _, _ = PM.particular_skewed_df1(coef, xg, dtype=np.float32)
    w2 = _df2_particular_f32(coef, xg)
    e1 = oracle.rel_err((w1 + corr).reshape(-1)[:n], y_ref)
    e2 = oracle.rel_err((w2 + corr).reshape(-1)[:n], y_ref)
    from scipy import signal
    s32 = np.hstack([sos[:, :3], np.ones((sos.shape[0], 1)), sos[:, 3:]]).astype(np.float32)
    e_seq = oracle.rel_err(signal.sosfilt(s32, x), y_ref)
    print(f"float32 error: sequential {e_seq:.2e}, direct-form-I order {e1:.2e}, direct form II {e2:.2e}")
    assert e1 <= 1.5 * e_seq
    assert e2 >= 2 * e1


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
