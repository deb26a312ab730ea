"""The library's host code on the CPU: sosfilt_api.cpp compiled against host stand-ins for the CUDA
runtime and the kernel launchers (tests/api_host/).

The stand-in launchers record each launch and, in place of the filter, write twice the input to the
output and add the samples processed to word 0 of the state.  That is enough to check, without a
GPU:

* the host precompute of the PH kernel (the float64 -> float32 tables): section constants, coupling blocks,
  lane and tile transition powers, the output basis and the input gain, against a float64
  derivation here from the transposed-direct-form-II recurrence (Eq. 1);
* which kernel a tuning selects, and the passes of a cascade of more than eight sections;
* the host-buffer pipeline of sos_filter_run_host: every sample passes through exactly one launch
  and the state is chained through the chunks, for ragged lengths and chunk sizes;
* the batched run's plan: one launch per (section count, b0 handling) class, each signal's tiles
  consecutive in the tile -> signal map, and each signal's buffers and length in its descriptor.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads
from paper_2607_23763_gb300._binding import Tuning
from workloads import designs

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_ROOT, "paper_2607_23763_gb300", "csrc")
_SRCS = [os.path.join(_HERE, "api_host", "api_host.cpp"), os.path.join(_CSRC, "sosfilt_api.cpp")]
_DEPS = _SRCS + [os.path.join(_HERE, "api_host", "cuda_runtime.h"), os.path.join(_ROOT, "include", "sosfilt.h"),
                 os.path.join(_CSRC, "sosfilt_internal.h")]
_LIB = os.path.join(_HERE, "_build", "libapi_host.so")
N64, W, C64 = 64, 7, 32 * 64
KIND_LANE, KIND_CASCADE, KIND_BATCH, KIND_SECTION, KIND_DTCR, KIND_TC = 1, 2, 3, 4, 5, 6


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not os.path.exists(_LIB) or any(os.path.getmtime(d) > os.path.getmtime(_LIB) for d in _DEPS):
        tmp = f"{_LIB}.{os.getpid()}.tmp"  # parallel test workers build side by side
        # -Bsymbolic: the library's own operator new calls bind to the harness's counting one
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-Wl,-Bsymbolic",
                        "-I", os.path.join(_HERE, "api_host"), "-I", os.path.join(_ROOT, "include"), "-I", _CSRC,
                        "-o", tmp, *_SRCS], check=True)
        os.replace(tmp, _LIB)
    L = ctypes.CDLL(_LIB)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sos_filter_create.argtypes = [c_int, vp, vp, vp, ctypes.POINTER(vp)]
    L.sos_filter_destroy.argtypes = [vp]
    L.sos_filter_run.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.sos_filter_run_host.argtypes = [vp, vp, vp, i64, vp, vp, i64]
    L.sos_filter_run_batch_ex.argtypes = [c_int, vp, vp, vp, vp, vp, vp, vp]
    L.host_launch.argtypes = [c_int, vp, ctypes.POINTER(ctypes.c_longlong), vp, ctypes.c_longlong]
    L.host_launch.restype = ctypes.c_longlong
    L.host_lane_layout.argtypes = [c_int, vp]
    L.host_lane_layout.restype = ctypes.c_longlong
    L.host_batch_layout.argtypes = [vp]
    return L


def _create(L, sos, tuning=None):
    sos = np.ascontiguousarray(sos, dtype=np.float64)
    h = ctypes.c_void_p()
    t = Tuning(**tuning) if tuning else None
    rc = L.sos_filter_create(sos.shape[0], sos.ctypes.data, None, None if t is None else ctypes.addressof(t),
                             ctypes.byref(h))
    assert rc == 0, rc
    return h


def _launches(L):
    out = []
    for i in range(L.host_launches()):
        info = (ctypes.c_int * 4)()
        grid = ctypes.c_longlong()
        size = L.host_launch(i, info, ctypes.byref(grid), None, 0)
        buf = (ctypes.c_ubyte * size)()
        L.host_launch(i, info, ctypes.byref(grid), buf, size)
        out.append({"kind": info[0], "K": info[1], "N": info[2], "norm": info[3], "grid": grid.value,
                    "raw": bytes(buf)})
    return out


def _at(raw, off, dtype, count=1):
    return np.frombuffer(raw, dtype=dtype, count=count, offset=off)


def _mem(addr, dtype, count):
    return np.ctypeslib.as_array((ctypes.c_byte * (np.dtype(dtype).itemsize * count)).from_address(addr)).view(dtype)


# ---------------------------------------------------------------- float64 derivations (Eq. 1)

def _normalised(sos):
    sos = np.asarray(sos, dtype=np.float64)
    norm = bool(np.all(sos[:, 0] != 0))
    c = sos.copy()
    if norm:
        c[:, 1] /= c[:, 0]
        c[:, 2] /= c[:, 0]
        c[:, 0] = 1.0
    return c, norm


def _step(c, z, x=0.0):
    """One sample through the cascade in transposed direct form II; z is updated in place."""
    v = x
    for k, (b0, b1, b2, a1, a2) in enumerate(c):
        y = b0 * v + z[2 * k]
        z[2 * k] = b1 * v - a1 * y + z[2 * k + 1]
        z[2 * k + 1] = b2 * v - a2 * y
        v = y
    return v


def _transition_and_basis(c, N):
    S = 2 * len(c)
    M1 = np.zeros((S, S))
    H = np.zeros((S, N))
    for j in range(S):
        z = np.zeros(S)
        z[j] = 1.0
        _step(c, z)
        M1[:, j] = z
        z = np.zeros(S)
        z[j] = 1.0
        for m in range(N):
            H[j, m] = _step(c, z)
    return M1, H


def _packed(M, K):
    out = []
    for s in range(K):
        for t in range(s + 1):
            out += [M[2 * s, 2 * t], M[2 * s, 2 * t + 1], M[2 * s + 1, 2 * t], M[2 * s + 1, 2 * t + 1]]
    return np.array(out)


def _close(got, want, what, seen=0.0):
    """float32 tables against float64 values: 2e-6 of the largest entry, plus float64 rounding of
    the products that formed them (1e-12 of `seen`, the largest intermediate entry)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    bound = 2e-6 * max(1e-30, float(np.abs(want).max())) + 1e-12 * seen
    err = float(np.abs(got - want).max())
    assert err <= bound, f"{what}: error {err:.3e} above {bound:.3e}"


# ---------------------------------------------------------------- tests

DESIGNS = {
    "butter2": designs.butter_lowpass(2, 0.2),
    "butter8": designs.butter_lowpass(8, 0.1),
    "butter16": designs.butter_lowpass(16, 0.05),
    "random5": designs.random_sections(workloads.uniform_f64(3, 15, stream=1).reshape(5, 3)),
    "resonators": designs.resonator_bank(),
}


@pytest.mark.parametrize("name", list(DESIGNS))
def test_ph_tables_match_a_float64_derivation(lib, name):
    sos = DESIGNS[name]
    K = sos.shape[0]
    f = _create(lib, sos)
    n = 3 * W * C64 + 5
    x = workloads.normal_f32(1, n)
    y = np.empty_like(x)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, n, None, None, None) == 0
    (l,) = _launches(lib)
    assert (l["kind"], l["K"], l["N"]) == (KIND_LANE, K, N64)
    offs = (ctypes.c_longlong * 21)()
    size = lib.host_lane_layout(K, offs)
    assert size == len(l["raw"])
    o = dict(zip(["x", "y", "n", "G", "n_tiles", "zi", "zf", "gain", "m_last", "tab", "sec", "MX", "A_tail"], offs))
    raw = l["raw"]
    G = -(-n // C64)
    assert _at(raw, o["n"], np.int64)[0] == n and _at(raw, o["G"], np.int64)[0] == G
    assert _at(raw, o["n_tiles"], np.int64)[0] == -(-G // W)
    assert _at(raw, o["x"], np.uint64)[0] == x.ctypes.data and _at(raw, o["y"], np.uint64)[0] == y.ctypes.data

    c, norm = _normalised(sos)
    assert bool(l["norm"]) == norm
    assert _at(raw, o["gain"], np.float32)[0] == pytest.approx(np.prod(sos[:, 0]) if norm else 1.0, rel=1e-6)
    M1, H = _transition_and_basis(c, N64)
    MN = np.linalg.matrix_power(M1, N64)
    AC = np.linalg.matrix_power(MN, 32)
    AT = np.linalg.matrix_power(AC, W)
    S = 2 * K
    # section constants (LaneSec: c, tn[5] as float4, then b0, zscale, zscale_inv, pad)
    sec = _at(raw, o["sec"], np.float32, 28 * K).reshape(K, 28)
    for j, (b0, b1, b2, a1, a2) in enumerate(c):
        _close(sec[j, 0:4], [b1, b2, -a1, -a2], f"{name} c[{j}]")
        P = MN[2 * j:2 * j + 2, 2 * j:2 * j + 2]
        for r in range(5):
            _close(sec[j, 4 + 4 * r:8 + 4 * r], P.reshape(-1), f"{name} tn[{j}][{r}]")
            P = P @ P
        zscale = np.prod(sos[j + 1:, 0]) if norm else 1.0
        _close(sec[j, 24:26], [b0, zscale], f"{name} b0, zscale[{j}]")
    # coupling blocks of M_N
    if K > 1:
        MX = _at(raw, o["MX"], np.float32, 2 * K * (K - 1)).reshape(-1, 4)
        for k in range(1, K):
            for j in range(k):
                _close(MX[k * (k - 1) // 2 + j], MN[2 * k:2 * k + 2, 2 * j:2 * j + 2].reshape(-1), f"{name} MX")
    # the table block: (M_N)^l and (A_T)^l packed, A_C, the basis H, A_T (column-major)
    nf = 2 * K * (K + 1)
    ms = nf if (nf // 4) % 2 else nf + 4
    full = S * S
    tab = _mem(int(_at(raw, o["tab"], np.uint64)[0]), np.float32, 64 * ms + 2 * full + N64 * S)
    # (the resonator bank's normalized sections couple with gains near 1e9, so the powers pass
    # through entries near 1e10 before they cancel: its float64 rounding is relative to those)
    Ml, Tl = np.eye(S), np.eye(S)
    seen_m = seen_t = 1.0
    for lane in range(32):
        seen_m, seen_t = max(seen_m, np.abs(Ml).max()), max(seen_t, np.abs(Tl).max())
        _close(tab[lane * ms:lane * ms + nf], _packed(Ml, K), f"{name} (M_N)^{lane}", seen_m)
        _close(tab[(32 + lane) * ms:(32 + lane) * ms + nf], _packed(Tl, K), f"{name} (A_T)^{lane}", seen_t)
        Ml, Tl = Ml @ MN, Tl @ AT
    off = 64 * ms
    _close(tab[off:off + full], AC.T.reshape(-1), f"{name} A_C")
    _close(tab[off + full:off + full + S * N64], H.reshape(-1), f"{name} basis")
    _close(tab[off + full + S * N64:off + 2 * full + S * N64], AT.T.reshape(-1), f"{name} A_T")
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("tuning,kind,N", [
    (None, KIND_LANE, 64), ({"N": 32}, KIND_LANE, 32), ({"deterministic": 1}, KIND_LANE, 64),
    ({"solver": 1}, KIND_CASCADE, 32), ({"solver": 1, "N": 64}, KIND_CASCADE, 64), ({"solver": 3}, KIND_DTCR, 64),
    ({"groups_per_cta": 10}, KIND_LANE, 64),
    ({"carry": 2, "N": 32}, KIND_SECTION, 32), ({"carry": 2, "N": 128}, KIND_SECTION, 128),
])
def test_a_tuning_selects_its_kernel(lib, tuning, kind, N):
    f = _create(lib, designs.butter_lowpass(8, 0.2), tuning)
    x = workloads.normal_f32(2, 50000)
    y = np.empty_like(x)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, x.size, None, None, None) == 0
    ls = _launches(lib)
    assert {(l["kind"], l["N"]) for l in ls} == {(kind, N)}
    np.testing.assert_array_equal(y, 2 * x * (1 if kind != KIND_SECTION else 2 ** (len(ls) - 1)))
    lib.sos_filter_destroy(f)


def test_more_than_eight_sections_run_in_passes(lib):
    sos = designs.random_sections(workloads.uniform_f64(5, 36, stream=1).reshape(12, 3))
    f = _create(lib, sos)
    x = workloads.normal_f32(3, 30000)
    y = np.empty_like(x)
    zi = np.arange(24, dtype=np.float32).reshape(12, 2)
    zf = np.zeros_like(zi)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, x.size, zi.ctypes.data, zf.ctypes.data, None) == 0
    ls = _launches(lib)
    assert [(l["kind"], l["K"]) for l in ls] == [(KIND_LANE, 8), (KIND_LANE, 4)]
    np.testing.assert_array_equal(y, 4 * x)  # the second pass filters the first one's output
    # each pass carries its own sections' states: word 0 of each pass's state advanced by n
    want = zi.copy()
    want[0, 0] += x.size
    want[8, 0] += x.size
    np.testing.assert_array_equal(zf, want)
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("n,chunk", [(0, 1000), (1, 1000), (999, 1000), (1000, 1000), (1001, 1000),
                                     (3 * 4096 + 5, 4096), (10007, 64), (20000, 20000 // 3)])
def test_run_host_passes_every_sample_once_and_chains_the_state(lib, n, chunk):
    f = _create(lib, designs.butter_lowpass(4, 0.2))
    x = workloads.normal_f32(4, n) if n else np.zeros(0, np.float32)
    y = np.full_like(x, np.nan)
    zi = np.array([[0.5, 1.0], [2.0, 3.0]], dtype=np.float32)
    zf = np.full_like(zi, np.nan)
    lib.host_reset()
    rc = lib.sos_filter_run_host(f, x.ctypes.data if n else None, y.ctypes.data if n else None, n,
                                 zi.ctypes.data, zf.ctypes.data, chunk)
    assert rc == 0
    np.testing.assert_array_equal(y, 2 * x)
    assert lib.host_launches() == -(-n // chunk)
    want = zi.copy()
    want[0, 0] += n
    np.testing.assert_array_equal(zf, want)
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("n", [0, 1, 5 * C64 + 3, 3 * W * C64 + 17])
def test_run_host_direct_is_one_run_on_the_host_buffers(lib, n):
    """chunk_samples = SOS_HOST_DIRECT: one run (one launch per pass) whose kernels take the host
    buffers' device mappings, the initial state in and the final state out; memory without a
    device mapping and overlapping buffers are rejected before any launch."""
    SOS_HOST_DIRECT = -1
    f = _create(lib, designs.butter_lowpass(4, 0.2))
    x = workloads.normal_f32(4, max(n, 1))[:n] if n else np.zeros(0, np.float32)
    y = np.full_like(x, np.nan)
    zi = np.array([[0.5, 1.0], [2.0, 3.0]], dtype=np.float32)
    zf = np.full_like(zi, np.nan)
    lib.host_reset()
    rc = lib.sos_filter_run_host(f, x.ctypes.data if n else None, y.ctypes.data if n else None, n,
                                 zi.ctypes.data, zf.ctypes.data, SOS_HOST_DIRECT)
    assert rc == 0
    ls = _launches(lib)
    assert len(ls) == (1 if n else 0)
    if n:
        offs = (ctypes.c_longlong * 21)()
        lib.host_lane_layout(2, offs)
        assert _at(ls[0]["raw"], offs[0], np.uint64)[0] == x.ctypes.data
        assert _at(ls[0]["raw"], offs[1], np.uint64)[0] == y.ctypes.data
    np.testing.assert_array_equal(y, 2 * x)
    want = zi.copy()
    want[0, 0] += n
    np.testing.assert_array_equal(zf, want)
    if n:
        lib.host_reset()
        assert lib.sos_filter_run_host(f, 16, y.ctypes.data, n, None, None, SOS_HOST_DIRECT) == -1
        if n > 1:
            assert lib.sos_filter_run_host(f, x.ctypes.data, x.ctypes.data + 4, n - 1, None, None, SOS_HOST_DIRECT) == -1
        assert lib.sos_filter_run_host(f, x.ctypes.data, y.ctypes.data, n, None, None, -2) == -1
        assert lib.host_launches() == 0
    lib.sos_filter_destroy(f)


def test_batched_plan_groups_signals_by_class_with_consecutive_tiles(lib):
    rng = np.random.default_rng(9)
    specs = []
    for i in range(40):
        K = [1, 2, 4, 8][i % 4]
        sos = designs.random_sections(workloads.uniform_f64(100 + i, 3 * K, stream=1).reshape(K, 3))
        if i % 5 == 0:
            sos[0, 0] = 0.0  # b0 = 0: the general (not normalized) class
        n = int(rng.choice([0, 1, 2047, 2048, 2049, 14336, 14337, 40000, 100003]))
        specs.append((sos, n))
    fs = [_create(lib, sos) for sos, _ in specs]
    xs = [workloads.normal_f32(200 + i, n) if n else np.zeros(1, np.float32) for i, (_, n) in enumerate(specs)]
    ys = [np.full_like(x, np.nan) for x in xs]
    zis = [np.full((sos.shape[0], 2), 0.25 * i, dtype=np.float32) for i, (sos, _) in enumerate(specs)]
    zfs = [np.full_like(z, np.nan) for z in zis]
    m = len(specs)
    arr = lambda vals: (ctypes.c_void_p * m)(*vals)
    lens = (ctypes.c_int64 * m)(*[n for _, n in specs])
    lib.host_reset()
    lib.host_batch_all_launches.restype = ctypes.c_longlong
    all_before = lib.host_batch_all_launches()
    rc = lib.sos_filter_run_batch_ex(m, arr([h.value for h in fs]), arr([x.ctypes.data for x in xs]),
                                     arr([y.ctypes.data for y in ys]), lens, arr([z.ctypes.data for z in zis]),
                                     arr([z.ctypes.data for z in zfs]), None)
    assert rc == 0
    lay = (ctypes.c_longlong * 17)()
    lib.host_batch_layout(lay)
    _, sig_size, ox, oy, on, oG, ot0, ozi, ozf, otab, ogain, p_sigs, p_tile_sig, p_ntiles, _, _, _ = lay
    launches = _launches(lib)
    # one persistent launch covers every class (recorded once per class)
    assert lib.host_batch_all_launches() - all_before == 1
    assert all(l["kind"] == KIND_BATCH for l in launches) and len({l["grid"] for l in launches}) == 1
    seen = []
    for l in launches:
        raw = l["raw"]
        n_tiles = int(_at(raw, p_ntiles, np.int64)[0])
        tile_sig = _mem(int(_at(raw, p_tile_sig, np.uint64)[0]), np.int32, n_tiles)
        n_sig = int(tile_sig.max()) + 1
        sigs = bytes(_mem(int(_at(raw, p_sigs, np.uint64)[0]), np.uint8, n_sig * sig_size))
        tiles = 0
        for k in range(n_sig):
            b = sigs[k * sig_size:(k + 1) * sig_size]
            i = next(j for j, x in enumerate(xs) if x.ctypes.data == _at(b, ox, np.uint64)[0])
            sos, n = specs[i]
            G = -(-n // C64)
            nt = -(-G // W)
            assert _at(b, on, np.int64)[0] == n and _at(b, oG, np.int64)[0] == G
            assert _at(b, oy, np.uint64)[0] == ys[i].ctypes.data
            assert _at(b, ozi, np.uint64)[0] == zis[i].ctypes.data and _at(b, ozf, np.uint64)[0] == zfs[i].ctypes.data
            t0 = int(_at(b, ot0, np.int64)[0])
            assert np.all(tile_sig[t0:t0 + nt] == k), i  # the signal's tiles are consecutive
            assert (l["K"], l["norm"]) == (sos.shape[0], int(np.all(sos[:, 0] != 0)))
            tiles += nt
            seen.append(i)
        assert tiles == n_tiles  # the map holds exactly the class's signals' tiles
    # every signal with samples is in exactly one class; the empty ones copy their state
    assert sorted(seen) == [i for i, (_, n) in enumerate(specs) if n > 0]  # once each
    for i, (sos, n) in enumerate(specs):
        if n:
            np.testing.assert_array_equal(ys[i], 2 * xs[i])
            want = zis[i].copy()
            want[0, 0] += n
            np.testing.assert_array_equal(zfs[i], want)
        else:
            np.testing.assert_array_equal(zfs[i], zis[i])
    for h in fs:
        lib.sos_filter_destroy(h)


@pytest.mark.parametrize("name", ["butter2", "butter16", "random5"])
@pytest.mark.parametrize("N", [32, 64, 128])
def test_cyclic_reduction_tables_match_the_float64_model(lib, name, N):
    """The per-section tables of the divide-and-conquer cyclic reduction (Eqs. 14-23) against the
    float64 step model, which the dense solves pin to the oracle."""
    from . import dccr_model as M
    sos = DESIGNS[name]
    K = sos.shape[0]
    f = _create(lib, sos, {"carry": 2, "N": N})
    x = workloads.normal_f32(5, 5 * 32 * N + 7)
    y = np.empty_like(x)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, x.size, None, None, None) == 0
    (l,) = _launches(lib)
    assert (l["kind"], l["K"], l["N"]) == (KIND_SECTION, K, N)
    lay = (ctypes.c_longlong * 18)()
    lib.host_pass_layout(lay)
    (sz, o_t0, o_b1, o_ne, o_f, o_nf, o_qo, o_qe, o_tn, o_tc, o_zs,
     p_sec, p_lane, p_grp, p_cta, p_nsec, p_gain, p_n) = lay
    raw = l["raw"]
    assert _at(raw, p_nsec, np.int32)[0] == K and _at(raw, p_n, np.int64)[0] == x.size
    c, norm = _normalised(sos)
    D = int(np.log2(N))
    lane_pow = _mem(int(_at(raw, p_lane, np.uint64)[0]), np.float32, K * 32 * 4).reshape(K, 32, 4)
    for k, (b0, b1, b2, a1, a2) in enumerate(c):
        sec = raw[p_sec + k * sz:p_sec + (k + 1) * sz]
        _close(_at(sec, o_t0, np.float32, 5), M.first_level_taps(b0, b1, b2, a1, a2), f"{name} taps[{k}]")
        _close(_at(sec, o_b1, np.float32, 4), [b1, b2, a1, a2], f"{name} b1 b2 a1 a2[{k}]")
        e, fl = M.level_coeffs(a1, a2, D)
        for i in range(1, D):
            _close(_at(sec, o_ne + 4 * i, np.float32), [-e[i]], f"{name} -e_{i}")
            _close(_at(sec, o_f + 4 * i, np.float32), [fl[i]], f"{name} f_{i}")
            _close(_at(sec, o_nf + 4 * i, np.float32), [-fl[i]], f"{name} -f_{i}")
        Q = M.q_tables(a1, a2, D)
        q = lambda lev, m: Q[lev][m] if 0 <= m < len(Q[lev]) else 0.0
        for lev in range(1, D + 1):
            mo, me = (1 << lev) - 1, (1 << lev) - 2
            _close(_at(sec, o_qo + 8 * lev, np.float32, 2), [q(lev, mo), q(lev, mo - 1)], f"{name} qo_{lev}")
            _close(_at(sec, o_qe + 8 * lev, np.float32, 2), [q(lev, me), q(lev, me - 1)], f"{name} qe_{lev}")
        T = M.transition(a1, a2)
        TN = np.linalg.matrix_power(T, N)
        P = TN
        for r in range(5):
            _close(_at(sec, o_tn + 16 * r, np.float32, 4), P.reshape(-1), f"{name} tn_{r}")
            P = P @ P
        Ll = np.eye(2)
        for lane in range(32):
            _close(lane_pow[k, lane], Ll.reshape(-1), f"{name} (T^N)^{lane}")
            Ll = Ll @ TN
        TC = Ll
        # group and block transitions for the per-section lookback: S^k (k <= 32), S^(32 i) (i <= 16)
        stride = 33 + 16 + 1
        for ptr, S in ((p_grp, TC), (p_cta, np.linalg.matrix_power(TC, 4))):
            pw = _mem(int(_at(raw, ptr, np.uint64)[0]), np.float32, K * stride * 4).reshape(K, stride, 4)[k]
            Pk = np.eye(2)
            for j in range(33):
                _close(pw[j], Pk.reshape(-1), f"{name} S^{j}")
                Pk = Pk @ S
            S32, P32 = np.linalg.matrix_power(S, 32), np.eye(2)
            for i in range(17):
                _close(pw[33 + i], P32.reshape(-1), f"{name} S^(32*{i})")
                P32 = P32 @ S32
        Wp = np.eye(2)
        for w in range(5):
            _close(_at(sec, o_tc + 16 * w, np.float32, 4), Wp.reshape(-1), f"{name} (T^C)^{w}")
            Wp = Wp @ TC
        zscale = np.prod(sos[k + 1:, 0]) if norm else 1.0
        _close(_at(sec, o_zs, np.float32), [zscale], f"{name} zscale[{k}]")
    lib.sos_filter_destroy(f)


def test_stream_push_continues_the_resident_state(lib):
    lib.sos_filter_stream_push.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_void_p]
    lib.sos_filter_stream_state.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    f = _create(lib, designs.butter_lowpass(6, 0.2))
    z_in = np.arange(6, dtype=np.float32).reshape(3, 2)
    assert lib.sos_filter_stream_state(f, None, z_in.ctypes.data, 0) == 0
    total = 0
    for n in (1, 2048, 14336 * 2 + 3, 0, 777):
        x = workloads.normal_f32(10 + n, n) if n else np.zeros(1, np.float32)
        y = np.full_like(x, np.nan)
        assert lib.sos_filter_stream_push(f, x.ctypes.data, y.ctypes.data, n, None) == 0
        if n:
            np.testing.assert_array_equal(y, 2 * x)
        total += n
    z = np.full((3, 2), np.nan, dtype=np.float32)
    assert lib.sos_filter_stream_state(f, z.ctypes.data, None, 0) == 0
    want = z_in.copy()
    want[0, 0] += total
    np.testing.assert_array_equal(z, want)
    lib.sos_filter_destroy(f)


def test_empty_run_copies_the_state_and_overlaps_are_rejected(lib):
    f = _create(lib, designs.butter_lowpass(4, 0.2))
    zi = np.array([[1.5, -2.0], [3.0, 4.0]], dtype=np.float32)
    zf = np.zeros_like(zi)
    lib.host_reset()
    assert lib.sos_filter_run(f, None, None, 0, zi.ctypes.data, zf.ctypes.data, None) == 0
    assert lib.host_launches() == 0
    np.testing.assert_array_equal(zf, zi)
    buf = workloads.normal_f32(6, 5000)
    # in place is allowed; a partial overlap is an argument error
    assert lib.sos_filter_run(f, buf.ctypes.data, buf.ctypes.data, 4000, None, None, None) == 0
    assert lib.sos_filter_run(f, buf.ctypes.data, buf.ctypes.data + 4 * 100, 4000, None, None, None) == -1
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("n", [1, 64, 65, 2047, 2048, 2049, 3 * 14336 + 100, 100003])
def test_final_state_tail_transition(lib, n):
    """For the final state the kernel needs the lane position of the last sample and the cascade's
    transition over the samples up to it: M1^(m_last + 1), recomputed when the position changes."""
    sos = DESIGNS["butter8"]
    K = sos.shape[0]
    f = _create(lib, sos)
    offs = (ctypes.c_longlong * 21)()
    lib.host_lane_layout(K, offs)
    o = dict(zip(["x", "y", "n", "G", "n_tiles", "zi", "zf", "gain", "m_last", "tab", "sec", "MX", "A_tail"], offs))
    c, _ = _normalised(sos)
    M1, _ = _transition_and_basis(c, 1)
    for length in (n, n + 1, n):  # a changed tail, then the first one again
        x = workloads.normal_f32(7, length)
        y = np.empty_like(x)
        zf = np.zeros((K, 2), dtype=np.float32)
        lib.host_reset()
        assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, length, None, zf.ctypes.data, None) == 0
        (l,) = _launches(lib)
        m_last = (length - 1) % N64  # groups are whole multiples of N samples
        assert _at(l["raw"], o["m_last"], np.int32)[0] == m_last
        want = _packed(np.linalg.matrix_power(M1, m_last + 1), K)
        _close(_at(l["raw"], o["A_tail"], np.float32, 2 * K * (K + 1)), want, f"tail n={length}")
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("name", ["butter2", "butter16", "random5"])
@pytest.mark.parametrize("N", [32, 64])
def test_cascade_carry_tables_match_a_float64_derivation(lib, name, N):
    """The whole-cascade carry of the cyclic-reduction kernel: lane and tile transition powers, A_C,
    A_T and its 32-tile powers for the lookback windows, and the output basis."""
    sos = DESIGNS[name]
    K = sos.shape[0]
    Wc = 8 if N == 32 else 4  # groups per tile of the cascade kernel
    f = _create(lib, sos, {"solver": 1, "N": N})
    x = workloads.normal_f32(8, 5 * Wc * 32 * N + 9)
    y = np.empty_like(x)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, x.size, None, None, None) == 0
    (l,) = _launches(lib)
    assert (l["kind"], l["K"], l["N"]) == (KIND_CASCADE, K, N)
    offs = (ctypes.c_longlong * 8)()
    assert lib.host_cas_layout(K, N, offs) == len(l["raw"])
    o_n, o_G, o_nt, o_gain, o_tab, o_sec, o_H, o_tail = offs
    raw = l["raw"]
    G = -(-x.size // (32 * N))
    assert _at(raw, o_G, np.int64)[0] == G and _at(raw, o_nt, np.int64)[0] == -(-G // Wc)
    c, _ = _normalised(sos)
    M1, H = _transition_and_basis(c, N)
    MN = np.linalg.matrix_power(M1, N)
    AC = np.linalg.matrix_power(MN, 32)
    AT = np.linalg.matrix_power(AC, Wc)
    S = 2 * K
    _close(_at(raw, o_H, np.float32, S * N), H.reshape(-1), f"{name} basis")
    nf = 2 * K * (K + 1)
    ms = nf if (nf // 4) % 2 else nf + 4
    full = S * S
    tab = _mem(int(_at(raw, o_tab, np.uint64)[0]), np.float32, 64 * ms + 18 * full)
    Ml, Tl = np.eye(S), np.eye(S)
    seen_m = seen_t = 1.0
    for lane in range(32):
        seen_m, seen_t = max(seen_m, np.abs(Ml).max()), max(seen_t, np.abs(Tl).max())
        _close(tab[lane * ms:lane * ms + nf], _packed(Ml, K), f"{name} (M_N)^{lane}", seen_m)
        _close(tab[(32 + lane) * ms:(32 + lane) * ms + nf], _packed(Tl, K), f"{name} (A_T)^{lane}", seen_t)
        Ml, Tl = Ml @ MN, Tl @ AT
    d = 64 * ms
    _close(tab[d:d + full], AC.T.reshape(-1), f"{name} A_C")
    _close(tab[d + full:d + 2 * full], AT.T.reshape(-1), f"{name} A_T")
    AT32 = np.linalg.matrix_power(AT, 32)
    Pw = AT32
    for w in range(1, 17):
        _close(tab[d + full * (1 + w):d + full * (2 + w)], Pw.T.reshape(-1), f"{name} (A_T)^(32*{w})")
        Pw = Pw @ AT32
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("N", [64, 32])
def test_batch_tables_match_a_float64_derivation(lib, N):
    """A signal of a batch carries its own tables for its tile geometry (N samples per lane, pinned
    here by the filter's tuning): the PH section constants and coupling blocks, the table block for
    tiles of seven groups, the gain, and the one-sample transition powers M1^(m+1), m < 64, from
    which the kernel forms a signal's final state."""
    sos = DESIGNS["butter8"]
    K = sos.shape[0]
    f = _create(lib, sos, {"N": N})
    x = workloads.normal_f32(12, 3 * W * 32 * N + 11)
    y = np.empty_like(x)
    zf = np.zeros((K, 2), dtype=np.float32)
    one = lambda v: (ctypes.c_void_p * 1)(v)
    lib.host_reset()
    assert lib.sos_filter_run_batch_ex(1, one(f.value), one(x.ctypes.data), one(y.ctypes.data),
                                       (ctypes.c_int64 * 1)(x.size), None, one(zf.ctypes.data), None) == 0
    (l,) = _launches(lib)
    assert (l["kind"], l["K"], l["N"]) == (KIND_BATCH, K, N)
    lay = (ctypes.c_longlong * 17)()
    lib.host_batch_layout(lay)
    sec_size, sig_size = lay[0], lay[1]
    otab, ogain, p_sigs, osec, oMX, oMm, oG = lay[9], lay[10], lay[11], lay[14], lay[15], lay[16], lay[5]
    sig = bytes(_mem(int(_at(l["raw"], p_sigs, np.uint64)[0]), np.uint8, sig_size))
    assert _at(sig, oG, np.int64)[0] == -(-x.size // (32 * N))  # groups of 32 N samples
    c, norm = _normalised(sos)
    M1, H = _transition_and_basis(c, N)
    MN = np.linalg.matrix_power(M1, N)
    AC = np.linalg.matrix_power(MN, 32)
    AT = np.linalg.matrix_power(AC, W)
    S, nf = 2 * K, 2 * K * (K + 1)
    assert _at(sig, ogain, np.float32)[0] == pytest.approx(np.prod(sos[:, 0]), rel=1e-6)
    secs = _mem(int(_at(sig, osec, np.uint64)[0]), np.float32, K * sec_size // 4).reshape(K, -1)
    for j, (b0, b1, b2, a1, a2) in enumerate(c):
        _close(secs[j, 0:4], [b1, b2, -a1, -a2], f"batch c[{j}]")
    MX = _mem(int(_at(sig, oMX, np.uint64)[0]), np.float32, 2 * K * (K - 1)).reshape(-1, 4)
    for k in range(1, K):
        for j in range(k):
            _close(MX[k * (k - 1) // 2 + j], MN[2 * k:2 * k + 2, 2 * j:2 * j + 2].reshape(-1), "batch MX")
    Mm = _mem(int(_at(sig, oMm, np.uint64)[0]), np.float32, N64 * nf).reshape(N64, nf)
    P = M1.copy()
    for m in range(N64):
        _close(Mm[m], _packed(P, K), f"batch M1^{m + 1}")
        P = P @ M1
    ms = nf if (nf // 4) % 2 else nf + 4
    full = S * S
    tab = _mem(int(_at(sig, otab, np.uint64)[0]), np.float32, 64 * ms + 2 * full + N * S)
    Ml, Tl = np.eye(S), np.eye(S)
    for lane in range(32):
        _close(tab[lane * ms:lane * ms + nf], _packed(Ml, K), f"batch (M_N)^{lane}")
        _close(tab[(32 + lane) * ms:(32 + lane) * ms + nf], _packed(Tl, K), f"batch (A_T)^{lane}")
        Ml, Tl = Ml @ MN, Tl @ AT
    _close(tab[64 * ms + full:64 * ms + full + S * N], H.reshape(-1), "batch basis")
    _close(tab[64 * ms + full + S * N:64 * ms + 2 * full + S * N], AT.T.reshape(-1), "batch A_T")
    lib.sos_filter_destroy(f)


def test_batch_plan_launches_reuse_the_uploaded_plan(lib):
    """A prepared plan uploads its signals once; every launch then runs one persistent launch over
    every (section count, b0 handling) class, on the same descriptors."""
    vp = ctypes.c_void_p
    lib.sos_batch_plan_create.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.sos_batch_plan_launch.argtypes = [vp, vp]
    lib.sos_batch_plan_status.argtypes = [vp]
    lib.sos_batch_plan_destroy.argtypes = [vp]
    specs = [(designs.butter_lowpass(2 * K, 0.2), n) for K, n in [(1, 5000), (4, 30000), (4, 777), (8, 60000)]]
    fs = [_create(lib, sos) for sos, _ in specs]
    xs = [workloads.normal_f32(300 + i, n) for i, (_, n) in enumerate(specs)]
    ys = [np.full_like(x, np.nan) for x in xs]
    m = len(specs)
    arr = lambda vals: (vp * m)(*vals)
    plan = vp()
    assert lib.sos_batch_plan_create(m, arr([h.value for h in fs]), arr([x.ctypes.data for x in xs]),
                                     arr([y.ctypes.data for y in ys]), (ctypes.c_int64 * m)(*[n for _, n in specs]),
                                     None, None, ctypes.byref(plan)) == 0
    for rep in range(2):
        lib.host_reset()
        for y in ys:
            y[:] = np.nan
        assert lib.sos_batch_plan_launch(plan, None) == 0
        ls = _launches(lib)
        assert sorted((l["kind"], l["K"]) for l in ls) == [(KIND_BATCH, 1), (KIND_BATCH, 4), (KIND_BATCH, 8)]
        assert len({l["grid"] for l in ls}) == 1  # the classes of one launch
        for x, y in zip(xs, ys):
            np.testing.assert_array_equal(y, 2 * x)
    assert lib.sos_batch_plan_status(plan) == 0
    assert lib.sos_batch_plan_destroy(plan) == 0
    for h in fs:
        lib.sos_filter_destroy(h)


def test_run_with_caller_scratch_allocates_nothing_and_checks_its_size(lib):
    """The path of sos_filter_run_noalloc: lookback descriptors and ticket counter in caller memory
    (the counter reset to zero for the launch, ticket base 0, the pass's descriptors cleared), a
    fresh epoch per pass, SOS_EBUDGET when the descriptors would not fit, and no call of an
    allocating runtime routine (cudaMalloc, cudaMallocHost, cudaFree, cudaFreeHost) nor of
    operator new during the run, with and without a final state."""
    lib.host_run_scratch.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_longlong, ctypes.c_void_p]
    sos = designs.random_sections(workloads.uniform_f64(21, 33, stream=1).reshape(11, 3))  # two passes
    f = _create(lib, sos)
    n = 5 * W * C64 + 3
    x = workloads.normal_f32(14, n)
    y = np.full_like(x, np.nan)
    n_tiles = -(-(-(-n // C64)) // W)
    need = n_tiles * 2 * 2 * 8
    where = (ctypes.c_ulonglong * 6)()
    lib.host_reset()
    assert lib.host_run_scratch(f, x.ctypes.data, y.ctypes.data, n, None, None, need - 1, where) == -6
    assert lib.host_launches() == 0
    # a run with a final state first: the tail transition for any length is prepared at creation
    zf = np.zeros((11, 2), np.float32)
    assert lib.host_run_scratch(f, x.ctypes.data, y.ctypes.data, n - 1, None, zf.ctypes.data, need, where) == 0
    assert (where[3], where[4], where[5]) == (0, 0, 0)
    lib.host_reset()
    assert lib.host_run_scratch(f, x.ctypes.data, y.ctypes.data, n, None, None, need, where) == 0
    assert where[3] == 0 and where[4] == 0  # no allocation of any kind
    assert where[5] == 0  # every descriptor word of the scratch was cleared before use
    np.testing.assert_array_equal(y, 4 * x)
    ls = _launches(lib)
    assert [l["K"] for l in ls] == [8, 3]
    epochs = []
    for l in ls:
        offs = (ctypes.c_longlong * 21)()
        lib.host_lane_layout(l["K"], offs)
        raw = l["raw"]
        assert _at(raw, offs[13], np.uint64)[0] == where[0] and _at(raw, offs[14], np.uint64)[0] == where[1]
        assert _at(raw, offs[15], np.uint64)[0] == 0
        epochs.append(int(_at(raw, offs[16], np.uint32)[0]))
    assert where[2] == 0  # the counter was reset for the launch
    assert len(set(epochs)) == 2 and all(e > 0 for e in epochs)
    lib.sos_filter_destroy(f)


def test_launch_parameters_follow_the_filter_settings(lib):
    """The wait budget, the phase-trace buffer, alignment, epochs and the ticket base that a launch
    receives come from the filter's settings and history."""
    lib.sos_filter_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    K = 4
    f = _create(lib, designs.butter_lowpass(2 * K, 0.2), {"spin_budget_cycles": 12345})
    trace = np.zeros((64, 32), dtype=np.uint64)
    assert lib.sos_filter_trace(f, trace.ctypes.data, 64) == 0
    n = 2 * W * C64 + 1
    x = workloads.normal_f32(15, n + 1)
    y = np.empty_like(x)
    offs = (ctypes.c_longlong * 21)()
    lib.host_lane_layout(K, offs)
    names = ["x", "y", "n", "G", "n_tiles", "zi", "zf", "gain", "m_last", "tab", "sec", "MX", "A_tail", "desc",
             "ticket", "ticket_base", "epoch", "spin_budget", "trace", "trace_tiles", "aligned"]
    o = dict(zip(names, offs))
    lib.host_reset()
    for src in (x, x[1:]):  # aligned, then 4 bytes off
        assert lib.sos_filter_run(f, src.ctypes.data, y.ctypes.data, n, None, None, None) == 0
    first, second = [l["raw"] for l in _launches(lib)]
    for raw in (first, second):
        assert _at(raw, o["spin_budget"], np.int64)[0] == 12345
        assert _at(raw, o["trace"], np.uint64)[0] == trace.ctypes.data and _at(raw, o["trace_tiles"], np.int64)[0] == 64
    assert _at(first, o["aligned"], np.int32)[0] == 1 and _at(second, o["aligned"], np.int32)[0] == 0
    # every launch has its own epoch; tickets continue from where the last launch left the counter
    assert _at(second, o["epoch"], np.uint32)[0] != _at(first, o["epoch"], np.uint32)[0]
    n_tiles = int(_at(first, o["n_tiles"], np.int64)[0])
    grid = _launches(lib)[0]["grid"]
    assert _at(second, o["ticket_base"], np.uint64)[0] == _at(first, o["ticket_base"], np.uint64)[0] + n_tiles + grid
    assert lib.sos_filter_trace(f, None, 0) == 0
    lib.sos_filter_destroy(f)


@pytest.mark.parametrize("tuning,kind,words_per_tile,W_tile", [(None, KIND_LANE, 4, 7), ({"solver": 1, "N": 64}, KIND_CASCADE, 2, 4),
                                                      ({"solver": 3}, KIND_DTCR, 2, 4)])
def test_a_captured_run_resets_its_own_counter_and_descriptors(lib, tuning, kind, words_per_tile, W_tile):
    """A run on a stream that is being captured into a CUDA graph takes the filter's second ticket
    counter, base 0 and the capture tag, and clears that counter and its descriptors first (inside the
    graph), leaving the eager launches' counter and ticket base as they were; it allocates nothing,
    so a run whose workspace would have to grow is refused during capture."""
    lib.host_set_capturing.argtypes = [ctypes.c_int]
    K = 4
    f = _create(lib, designs.butter_lowpass(2 * K, 0.2), tuning)
    N = 64
    n = 3 * W_tile * 32 * N + 5
    x = workloads.normal_f32(16, n)
    y = np.empty_like(x)
    offs = (ctypes.c_longlong * 21)()
    lib.host_lane_layout(K, offs)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, n, None, None, None) == 0  # eager: workspace
    (eager,) = _launches(lib)
    if kind == KIND_LANE:
        o_desc, o_ticket, o_base, o_epoch = offs[13], offs[14], offs[15], offs[16]
    else:
        c_offs = (ctypes.c_longlong * 8)()
        lib.host_cas_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.host_cas_layout(K, N, c_offs)
        # CasParams: x, y, n, G, n_tiles, zi, zf, gain, desc, ticket, ticket_base, epoch
        o_desc = 8 * 7 + 8
        o_ticket, o_base, o_epoch = o_desc + 8, o_desc + 16, o_desc + 24
    t_eager = int(_at(eager["raw"], o_ticket, np.uint64)[0])
    base_eager = int(_at(eager["raw"], o_base, np.uint64)[0])
    desc = int(_at(eager["raw"], o_desc, np.uint64)[0])
    n_tiles = -(-(-(-n // (32 * N))) // W_tile)
    used = _mem(desc, np.uint64, n_tiles * words_per_tile * K)
    used[:] = 0xabab  # stale words left by earlier launches
    _mem(t_eager + 8, np.uint64, 1)[:] = 777  # the captured counter's stale value
    lib.host_set_capturing(1)
    try:
        lib.host_reset()
        assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, n, None, None, None) == 0
        (cap,) = _launches(lib)
        assert int(_at(cap["raw"], o_ticket, np.uint64)[0]) == t_eager + 8
        assert int(_at(cap["raw"], o_base, np.uint64)[0]) == 0
        assert int(_at(cap["raw"], o_epoch, np.uint32)[0]) == 0x3fffffff
        assert np.all(used == 0) and _mem(t_eager + 8, np.uint64, 1)[0] == 0
        # no allocation while capturing: a longer signal than the workspace holds is refused
        big = np.zeros(2048 * 32 * N, np.float32)  # 2048 groups: more than the workspace holds
        assert lib.sos_filter_run(f, big.ctypes.data, big.ctypes.data, big.size, None, None, None) == -1
    finally:
        lib.host_set_capturing(0)
    lib.host_reset()
    assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, n, None, None, None) == 0  # eager again
    (again,) = _launches(lib)
    assert int(_at(again["raw"], o_ticket, np.uint64)[0]) == t_eager
    assert int(_at(again["raw"], o_base, np.uint64)[0]) == base_eager + n_tiles + eager["grid"]
    lib.sos_filter_destroy(f)


def _tune_costs(lib, fastest):
    """Simulated launch times: the candidate fastest(K) takes 1 ms per launch, the others 2 and 3."""
    cands = [(KIND_CASCADE, 32), (KIND_CASCADE, 64), (KIND_LANE, 64), (KIND_DTCR, 64), (KIND_TC, 64)]  # the autotuner's candidates
    # (the PH candidates with 7 and 10 groups per tile are both (KIND_LANE, 64) here: equal simulated times,
    # and the first measured of them, 7 groups, is kept)
    for K in range(1, 9):
        best = fastest(K)
        slow = 2.0
        for c in cands:
            lib.host_set_cost(c[0], c[1], K, 1.0 if c == best else slow)
            slow += 0.0 if c == best else 1.0


def test_autotuner_choices_drive_the_default_launch(lib):
    """The autotuner times its candidates per section count and length bucket and keeps the fastest;
    default-tuned runs then launch that choice, an explicit tuning still wins."""
    lib.sos_autotune.argtypes = [ctypes.c_int, ctypes.c_void_p]
    lib.sos_autotune_choice.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
    lib.host_set_cost.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float]
    solver, N = ctypes.c_int(), ctypes.c_int()

    def choice(K, n):
        assert lib.sos_autotune_choice(K, n, ctypes.byref(solver), ctypes.byref(N)) == 0
        return solver.value, N.value

    assert choice(4, 1 << 20) == (0, 0)  # nothing tuned yet: the library's defaults
    report = np.zeros((8, 4, 6), dtype=np.float32)
    fastest = {5: (KIND_DTCR, 64), 7: (KIND_TC, 64)}
    _tune_costs(lib, lambda K: (KIND_CASCADE, 32) if K <= 3 else fastest.get(K, (KIND_LANE, 64)))
    lib.host_set_light(1)
    try:
        assert lib.sos_autotune(16, report.ctypes.data) == 0
    finally:
        lib.host_set_light(0)
    for K in range(1, 9):
        want = (1, 32) if K <= 3 else (3, 64) if K == 5 else (4, 64) if K == 7 else (2, 64)
        for n in (1000, 1 << 16, 1 << 22, 1 << 30):  # buckets above 2^16 repeat the measured one
            assert choice(K, n) == want, (K, n)
        assert np.argmax(report[K - 1, 0]) == (0 if K <= 3 else 3 if K == 5 else 5 if K == 7 else 2)
        np.testing.assert_array_equal(report[K - 1, 1:], np.repeat(report[K - 1, :1], 3, axis=0))
    assert choice(12, 1 << 20) == (2, 64)  # more than eight sections: the eight-section choice

    x = workloads.normal_f32(13, 40000)
    y = np.empty_like(x)
    for K, tuning, want in [(2, None, (KIND_CASCADE, 32)), (6, None, (KIND_LANE, 64)), (5, None, (KIND_DTCR, 64)),
                            (7, None, (KIND_TC, 64)), (2, {"solver": 2}, (KIND_LANE, 64)),
                            (2, {"solver": 3}, (KIND_DTCR, 64)), (2, {"solver": 4}, (KIND_TC, 64))]:
        f = _create(lib, designs.butter_lowpass(2 * K, 0.2), tuning)
        lib.host_reset()
        assert lib.sos_filter_run(f, x.ctypes.data, y.ctypes.data, x.size, None, None, None) == 0
        assert {(l["kind"], l["N"]) for l in _launches(lib)} == {want}, (K, tuning)
        lib.sos_filter_destroy(f)

    # leave the library tuned to its untuned defaults (PH, N = 64) for the tests after this one
    _tune_costs(lib, lambda K: (KIND_LANE, 64))
    lib.host_set_light(1)
    try:
        assert lib.sos_autotune(16, None) == 0
    finally:
        lib.host_set_light(0)
        lib.host_reset()


def test_batch_autotuner_picks_the_tile_geometry_per_section_count(lib):
    """The batch autotuner times both tile geometries per section count and signal length from
    prepared plans and keeps the faster; default-tuned batched runs then put each signal in the
    class of its geometry (tiles of 32 N samples per group), a filter's tuning N still wins, and one
    persistent launch covers the mix."""
    vp = ctypes.c_void_p
    lib.sos_autotune_batch.argtypes = [vp]
    lib.sos_autotune_batch_choice.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    lib.host_set_cost.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float]
    lib.host_batch_all_launches.restype = ctypes.c_longlong
    N = ctypes.c_int()

    def choice(K, n):
        assert lib.sos_autotune_batch_choice(K, n, ctypes.byref(N)) == 0
        return N.value

    def tune(fast32):
        for K in range(1, 9):
            lib.host_set_cost(KIND_BATCH, 32, K, 1.0 if fast32(K) else 2.0)
            lib.host_set_cost(KIND_BATCH, 64, K, 2.0 if fast32(K) else 1.0)
        report = np.zeros((8, 4, 2), dtype=np.float32)
        lib.host_set_light(1)
        try:
            assert lib.sos_autotune_batch(report.ctypes.data) == 0
        finally:
            lib.host_set_light(0)
            lib.host_reset()
        return report

    report = tune(lambda K: K <= 4)
    for K in range(1, 9):
        assert np.all(report[K - 1, :, 1] > 0) and np.all(report[K - 1, :, 0] > 0)
        assert np.all(np.argmax(report[K - 1], axis=1) == (1 if K <= 4 else 0)), K
        for n in (1000, 1 << 15, 1 << 20, 1 << 30):
            assert choice(K, n) == (32 if K <= 4 else 64), (K, n)
    assert choice(12, 1 << 20) == 64  # more than eight sections: the eight-section choice
    try:
        specs = [(2, None, 32), (2, {"N": 64}, 64), (8, None, 64), (8, {"N": 32}, 32), (4, None, 32)]
        fs = [_create(lib, designs.butter_lowpass(2 * K, 0.2), t) for K, t, _ in specs]
        n = 3 * W * C64 + 5
        xs = [workloads.normal_f32(40 + i, n) for i in range(len(specs))]
        ys = [np.empty_like(x) for x in xs]
        m = len(specs)
        arr = lambda vals: (vp * m)(*vals)
        lib.host_reset()
        before = lib.host_batch_all_launches()
        assert lib.sos_filter_run_batch_ex(m, arr([h.value for h in fs]), arr([x.ctypes.data for x in xs]),
                                           arr([y.ctypes.data for y in ys]), (ctypes.c_int64 * m)(*[n] * m), None,
                                           None, None) == 0
        assert lib.host_batch_all_launches() - before == 1
        lay = (ctypes.c_longlong * 17)()
        lib.host_batch_layout(lay)
        sig_size, ox, oG, p_sigs, p_ntiles = lay[1], lay[2], lay[5], lay[11], lay[13]
        got = {}
        for l in _launches(lib):
            n_tiles = int(_at(l["raw"], p_ntiles, np.int64)[0])
            tile_sig = _mem(int(_at(l["raw"], lay[12], np.uint64)[0]), np.int32, n_tiles)
            n_sig = int(tile_sig.max()) + 1
            sigs = bytes(_mem(int(_at(l["raw"], p_sigs, np.uint64)[0]), np.uint8, n_sig * sig_size))
            for k in range(n_sig):
                b = sigs[k * sig_size:(k + 1) * sig_size]
                i = next(j for j, x in enumerate(xs) if x.ctypes.data == _at(b, ox, np.uint64)[0])
                G = -(-n // (32 * l["N"]))
                assert _at(b, oG, np.int64)[0] == G
                got[i] = (l["K"], l["N"], n_tiles)
        for i, (K, _, Nw) in enumerate(specs):
            assert got[i][:2] == (K, Nw), i
            np.testing.assert_array_equal(ys[i], 2 * xs[i])
        # the two eight-section signals sit in different classes, each with its own tiles
        assert got[2][2] == -(-(-(-n // C64)) // W) and got[3][2] == -(-(-(-n // (32 * 32))) // W)
        for h in fs:
            lib.sos_filter_destroy(h)
    finally:
        tune(lambda K: False)  # leave the library's batched runs at N = 64 for the other tests
