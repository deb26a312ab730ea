"""Host-thread emulation of the PH kernels' lookback protocol (tests/lookback_emu.c).

Worker threads draw tiles from an ascending ticket counter, publish tagged local carries, compose
each tile's incoming state from its anchor's resolved carry and the local carries after it with
bounded spins, and publish resolved carries at anchors.  The tests check that any interleaving
gives the single-thread result bit for bit, that stale tags of an earlier launch over the same
descriptor memory are never taken, and that a tile which never publishes makes its successors'
waits run out and return (no hang) with the status set.  The tensor-core kernel's hierarchical
form (anchors every 32 tiles post their local part early, super-anchors every 128 tiles chain the
resolved carries) is checked the same way, and against the recurrence in float64.  The batched form shares one ticket queue
among the tiles of several signals, each signal with its own chain, anchors and transition, as the
batch kernel does.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lookback_emu.c")
_LIB = os.path.join(_HERE, "_build", "liblookback_emu.so")


@pytest.fixture(scope="module")
def emu():
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = f"{_LIB}.{os.getpid()}.tmp"  # parallel test workers build side by side
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    lib = ctypes.CDLL(_LIB)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.emu_run.argtypes = [ctypes.c_int, i64, ctypes.c_uint, vp, vp, vp, vp, vp, ctypes.c_int, i64, i64]
    lib.emu_run.restype = ctypes.c_int
    lib.emu_reference.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp]
    lib.emu_run_batch.argtypes = [ctypes.c_int, i64, ctypes.c_uint, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, i64, i64]
    lib.emu_run_batch.restype = ctypes.c_int
    lib.emu_reference_batch.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp]
    lib.emu_run_hier.argtypes = [ctypes.c_int, i64, ctypes.c_uint, vp, vp, vp, vp, vp, vp, ctypes.c_int, i64, i64]
    lib.emu_run_hier.restype = ctypes.c_int
    lib.emu_reference_hier.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp]
    return lib


def _case(S, n_tiles, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((S, S)).astype(np.float32)
    A *= np.float32(0.9 / max(1e-6, np.abs(np.linalg.eigvals(A.astype(np.float64))).max()))
    local = rng.standard_normal((n_tiles, S)).astype(np.float32)
    z0 = rng.standard_normal(S).astype(np.float32)
    return np.ascontiguousarray(A), local, z0


def _p(a):
    return a.ctypes.data


@pytest.mark.parametrize("S,n_tiles,threads", [(2, 1, 4), (4, 33, 3), (16, 200, 8), (16, 97, 1), (6, 64, 16)])
def test_any_interleaving_gives_the_serial_result(emu, S, n_tiles, threads):
    A, local, z0 = _case(S, n_tiles, S * 1000 + n_tiles)
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference(S, n_tiles, _p(local), _p(A), _p(z0), _p(ref))
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    for epoch in (1, 2, 3):  # the same descriptor memory, launch after launch
        Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
        rc = emu.emu_run(S, n_tiles, epoch, _p(desc), _p(local), _p(A), _p(z0), _p(Z), threads, 1 << 22, -1)
        assert rc == 0
        assert np.array_equal(Z, ref)


def test_stale_tags_of_an_earlier_launch_are_not_taken(emu):
    # a launch over different carries leaves tagged words behind; the next launch, with the next
    # epoch, must not compose any of them
    S, n_tiles = 8, 150
    A, local, z0 = _case(S, n_tiles, 7)
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    other = (local * 3 + 1).astype(np.float32)
    Z = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run(S, n_tiles, 5, _p(desc), _p(other), _p(A), _p(z0), _p(Z), 6, 1 << 22, -1) == 0
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference(S, n_tiles, _p(local), _p(A), _p(z0), _p(ref))
    Z2 = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run(S, n_tiles, 6, _p(desc), _p(local), _p(A), _p(z0), _p(Z2), 6, 1 << 22, -1) == 0
    assert np.array_equal(Z2, ref)


@pytest.mark.parametrize("silent", [0, 5, 32, 40])
def test_a_tile_that_never_publishes_times_out_its_successors(emu, silent):
    S, n_tiles = 4, 120
    A, local, z0 = _case(S, n_tiles, 11)
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference(S, n_tiles, _p(local), _p(A), _p(z0), _p(ref))
    Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
    rc = emu.emu_run(S, n_tiles, 1, _p(desc), _p(local), _p(A), _p(z0), _p(Z), 4, 2000, silent)
    assert rc == 1  # the waits ran out and every worker returned
    # tiles before the silent one never depended on it
    assert np.array_equal(Z[:silent], ref[:silent])


def _batch_case(S, sig_tiles, seed):
    rng = np.random.default_rng(seed)
    n_sig = len(sig_tiles)
    AT = np.empty((n_sig, S, S), dtype=np.float32)
    for k in range(n_sig):
        A = rng.standard_normal((S, S))
        AT[k] = (A * (0.9 / max(1e-6, np.abs(np.linalg.eigvals(A)).max()))).astype(np.float32)
    tile0 = np.concatenate([[0], np.cumsum(sig_tiles)[:-1]]).astype(np.int64)
    n_tiles = int(np.sum(sig_tiles))
    tile_sig = np.repeat(np.arange(n_sig, dtype=np.int32), sig_tiles)
    local = rng.standard_normal((n_tiles, S)).astype(np.float32)
    z0 = rng.standard_normal((n_sig, S)).astype(np.float32)
    return AT, tile0, np.asarray(sig_tiles, dtype=np.int64), n_tiles, tile_sig, local, z0


@pytest.mark.parametrize("S,sig_tiles,threads", [
    (4, [1, 31, 32, 33, 65, 1, 64], 6),
    (16, [97, 3, 40], 8),
    (2, [1] * 50, 4),
    (8, [200], 1),
])
def test_batched_chains_give_each_signal_its_serial_result(emu, S, sig_tiles, threads):
    AT, tile0, nst, n_tiles, tile_sig, local, z0 = _batch_case(S, sig_tiles, S + len(sig_tiles))
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference_batch(S, len(sig_tiles), _p(tile0), _p(nst), _p(local), _p(AT), _p(z0), _p(ref))
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    for epoch in (1, 2):
        Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
        rc = emu.emu_run_batch(S, n_tiles, epoch, _p(desc), _p(local), _p(AT), _p(z0), _p(tile_sig), _p(tile0),
                               _p(Z), threads, 1 << 22, -1)
        assert rc == 0
        assert np.array_equal(Z, ref)
    # each signal's chain is the single-signal protocol on its own tiles
    for k, (t0, nt) in enumerate(zip(tile0, nst)):
        one = np.zeros((nt, S), dtype=np.float32)
        emu.emu_reference(S, int(nt), _p(np.ascontiguousarray(local[t0:t0 + nt])), _p(np.ascontiguousarray(AT[k])),
                          _p(np.ascontiguousarray(z0[k])), _p(one))
        assert np.array_equal(ref[t0:t0 + nt], one), k


def test_batched_chains_do_not_cross_signals(emu):
    """The first tile of every signal starts from that signal's own initial state, whatever the tile
    before it in the queue holds; changing one signal's carries changes no other signal's result."""
    S, sig_tiles = 4, [33, 20, 70]
    AT, tile0, nst, n_tiles, tile_sig, local, z0 = _batch_case(S, sig_tiles, 3)
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    Z1 = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run_batch(S, n_tiles, 1, _p(desc), _p(local), _p(AT), _p(z0), _p(tile_sig), _p(tile0),
                             _p(Z1), 5, 1 << 22, -1) == 0
    local2 = local.copy()
    local2[tile0[1]:tile0[1] + nst[1]] *= 7  # only the second signal's carries
    Z2 = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run_batch(S, n_tiles, 2, _p(desc), _p(local2), _p(AT), _p(z0), _p(tile_sig), _p(tile0),
                             _p(Z2), 5, 1 << 22, -1) == 0
    s1 = slice(tile0[1], tile0[1] + nst[1])
    assert np.array_equal(np.delete(Z1, np.r_[s1], axis=0), np.delete(Z2, np.r_[s1], axis=0))
    assert not np.array_equal(Z1[s1][1:], Z2[s1][1:])
    for k in range(3):
        assert np.array_equal(Z1[tile0[k]], z0[k])


def test_batched_silent_tile_times_out_only_later_work(emu):
    S, sig_tiles = 4, [40, 50, 30]
    AT, tile0, nst, n_tiles, tile_sig, local, z0 = _batch_case(S, sig_tiles, 9)
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference_batch(S, 3, _p(tile0), _p(nst), _p(local), _p(AT), _p(z0), _p(ref))
    silent = int(tile0[1] + 5)
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
    rc = emu.emu_run_batch(S, n_tiles, 1, _p(desc), _p(local), _p(AT), _p(z0), _p(tile_sig), _p(tile0), _p(Z),
                           4, 2000, silent)
    assert rc == 1
    assert np.array_equal(Z[:silent], ref[:silent])  # the first signal and the silent tile's predecessors


def _powers(A):
    """A^k, k = 0 .. 32, float32 (from float64 products)."""
    S = A.shape[0]
    P = np.empty((33, S, S), dtype=np.float32)
    M = np.eye(S)
    for k in range(33):
        P[k] = M
        M = M @ A.astype(np.float64)
    return np.ascontiguousarray(P)


@pytest.mark.parametrize("S,n_tiles,threads", [(2, 1, 4), (4, 33, 3), (16, 300, 8), (6, 129, 1), (8, 520, 16),
                                               (4, 128, 5), (4, 161, 6)])
def test_hierarchical_any_interleaving_gives_the_serial_result(emu, S, n_tiles, threads):
    A, local, z0 = _case(S, n_tiles, S * 100 + n_tiles)
    AP = _powers(A)
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference_hier(S, n_tiles, _p(local), _p(A), _p(AP), _p(z0), _p(ref))
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    for epoch in (1, 2, 3):
        Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
        rc = emu.emu_run_hier(S, n_tiles, epoch, _p(desc), _p(local), _p(A), _p(AP), _p(z0), _p(Z), threads,
                              1 << 22, -1)
        assert rc == 0
        assert np.array_equal(Z, ref)
    # the composition is the recurrence Z(t + 1) = A Z(t) + L(t), up to float32 rounding
    z = z0.astype(np.float64)
    want = np.empty((n_tiles, S))
    for t in range(n_tiles):
        want[t] = z
        z = A.astype(np.float64) @ z + local[t]
    assert np.allclose(ref, want, rtol=1e-4, atol=1e-4 * np.abs(want).max())


def test_hierarchical_stale_tags_are_not_taken(emu):
    S, n_tiles = 8, 300
    A, local, z0 = _case(S, n_tiles, 17)
    AP = _powers(A)
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    other = (local * 3 + 1).astype(np.float32)
    Z = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run_hier(S, n_tiles, 5, _p(desc), _p(other), _p(A), _p(AP), _p(z0), _p(Z), 6, 1 << 22, -1) == 0
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference_hier(S, n_tiles, _p(local), _p(A), _p(AP), _p(z0), _p(ref))
    Z2 = np.zeros((n_tiles, S), dtype=np.float32)
    assert emu.emu_run_hier(S, n_tiles, 6, _p(desc), _p(local), _p(A), _p(AP), _p(z0), _p(Z2), 6, 1 << 22, -1) == 0
    assert np.array_equal(Z2, ref)


@pytest.mark.parametrize("silent", [0, 5, 32, 128, 140])
def test_hierarchical_silent_tile_times_out_its_successors(emu, silent):
    S, n_tiles = 4, 300
    A, local, z0 = _case(S, n_tiles, 19)
    AP = _powers(A)
    ref = np.zeros((n_tiles, S), dtype=np.float32)
    emu.emu_reference_hier(S, n_tiles, _p(local), _p(A), _p(AP), _p(z0), _p(ref))
    desc = np.zeros(n_tiles * 2 * S, dtype=np.uint64)
    Z = np.full((n_tiles, S), np.nan, dtype=np.float32)
    rc = emu.emu_run_hier(S, n_tiles, 1, _p(desc), _p(local), _p(A), _p(AP), _p(z0), _p(Z), 4, 2000, silent)
    assert rc == 1
    assert np.array_equal(Z[:silent], ref[:silent])
