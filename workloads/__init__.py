"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the benchmark.

This module draws numbers and designs filters; it holds none of the filtering
arithmetic of the method.  Everything is a deterministic function of a seed:

* signals: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller, float32
  (``normal_f32``); the C generator in ``philox_gen.c`` is the fast path and
  ``philox4x32_10_np`` is an independent numpy restatement used to test it;
* filter designs (``designs``): Butterworth low-pass in second-order
  sections through the bilinear transform (the paper's benchmark filters,
  Sec. IV-F), a narrow-band resonator bank at pole radius 0.999 (precision
  stress), and random stable sections (batched and serving mixes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import designs  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "philox_gen.c")
_LIB_PATH = os.path.join(_HERE, "_libsosinputs.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared library (plain gcc, no arch flags)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.wl_normal_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.wl_normal_f32.restype = ctypes.c_int
            lib.wl_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_int]
            lib.wl_uniform_f64.restype = ctypes.c_int
            lib.wl_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.wl_philox4x32_10.restype = None
            _lib = lib
    return _lib


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def normal_f32(seed: int, n: int, stream: int = 0, sin_amp: float = 0.0, sin_omega: float = 0.0,
               out: np.ndarray | None = None) -> np.ndarray:
    """n float32 samples of N(0,1) from (seed, stream); optionally plus sin_amp*sin(sin_omega*k)."""
    lib = _load()
    if out is None:
        out = np.empty(n, dtype=np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size >= n
    if n:
        lib.wl_normal_f32(seed, stream, n, out.ctypes.data, float(sin_amp), float(sin_omega), _threads())
    return out


def uniform_f64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles uniform in (0,1) from (seed, stream)."""
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    if n:
        lib.wl_uniform_f64(seed, stream, n, out.ctypes.data, _threads())
    return out


# ---------------------------------------------------------------------------
# Mixes of many signals (batched runs) and many streams (serving).

BATCH_ORDERS = (2, 4, 8, 16)
SERVE_ORDERS = (2, 4, 8, 16)
SERVE_ORDER_SHARES = (0.40, 0.30, 0.20, 0.10)


def batched_signal(i: int, seed_base: int = 1000, log2_min: float = 10.0, log2_max: float = 22.0):
    """Signal i of the batched mix: (sos, length, input seed).

    Order uniform over {2, 4, 8, 16}; length round(2^U) with U uniform in [log2_min, log2_max];
    random stable sections (``designs.random_sections``); input N(0,1) from seed seed_base + i.
    """
    u = uniform_f64(seed_base + i, 2 + 3 * 8, stream=1)
    order = BATCH_ORDERS[min(3, int(u[0] * 4))]
    n = int(round(2.0 ** (log2_min + (log2_max - log2_min) * u[1])))
    K = order // 2
    sos = designs.random_sections(u[2:2 + 3 * K].reshape(K, 3))
    return sos, n, seed_base + i


def serving_stream(sid: int, seed_base: int = 500000):
    """Stream sid of the serving mix: sos with order 2/4/8/16 at 40/30/20/10 %, random sections."""
    u = uniform_f64(seed_base + sid, 1 + 3 * 8, stream=2)
    c = np.cumsum(SERVE_ORDER_SHARES)
    order = SERVE_ORDERS[int(np.searchsorted(c, u[0], side="right"))]
    K = order // 2
    return designs.random_sections(u[1:1 + 3 * K].reshape(K, 3))


def serving_chunk_len(sid: int, chunk: int, seed_base: int = 500000, lo: int = 4096, hi: int = 65536) -> int:
    """Length of chunk `chunk` of stream sid: uniform integer in [lo, hi]."""
    u = uniform_f64(seed_base + sid, 1, stream=(3 << 32) + chunk)[0]
    return lo + min(hi - lo, int(u * (hi - lo + 1)))


def serving_chunk(sid: int, chunk: int, n: int, seed_base: int = 500000) -> np.ndarray:
    """Input of chunk `chunk` of stream sid: n samples of N(0,1)."""
    return normal_f32(seed_base + sid, n, stream=(4 << 32) + chunk)


def philox4x32_10_c(ctr, key) -> list[int]:
    """One Philox4x32-10 block through the C generator (for known-answer tests)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.wl_philox4x32_10(ctypes.addressof(c), ctypes.addressof(k), ctypes.addressof(o))
    return list(o)


# ---------------------------------------------------------------------------
# Independent numpy restatement (vectorised over blocks), used to test the C path.
_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on uint32 arrays (broadcast); returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint32) + np.zeros_like(c0)
    k1 = np.asarray(k1, dtype=np.uint32) + np.zeros_like(c0)
    for r in range(10):
        if r:
            k0 = (k0 + _W0).astype(np.uint32)
            k1 = (k1 + _W1).astype(np.uint32)
        p0 = _M0 * c0.astype(np.uint64)
        p1 = _M1 * c2.astype(np.uint64)
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & _MASK).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & _MASK).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform_f64_np(seed: int, n: int, stream: int = 0) -> np.ndarray:
    nb = (n + 1) // 2
    i = np.arange(nb, dtype=np.uint64)
    o0, o1, o2, o3 = philox4x32_10_np((i & _MASK).astype(np.uint32), (i >> np.uint64(32)).astype(np.uint32),
                                      np.uint32(stream & 0xFFFFFFFF), np.uint32(stream >> 32),
                                      np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32))
    w0 = (o1.astype(np.uint64) << np.uint64(32)) | o0.astype(np.uint64)
    w1 = (o3.astype(np.uint64) << np.uint64(32)) | o2.astype(np.uint64)
    u0 = ((w0 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u1 = ((w1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return np.stack([u0, u1], axis=1).reshape(-1)[:n]


def normal_f32_np(seed: int, n: int, stream: int = 0) -> np.ndarray:
    u = uniform_f64_np(seed, 2 * ((n + 1) // 2), stream).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    z = np.stack([r * np.cos(2 * np.pi * u[:, 1]), r * np.sin(2 * np.pi * u[:, 1])], axis=1)
    return z.reshape(-1)[:n].astype(np.float32)
