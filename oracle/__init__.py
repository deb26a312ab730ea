"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct float64 CPU implementation of what the GPU
library computes: the cascade of second-order sections of Eq. 1 (Sec. II-A),
evaluated sample by sample in the transposed direct form II (see
``sosfilt_oracle.c``).  It shares no code with the GPU library; only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it.

Pins (tests/test_oracle_pins.py) tie it to the mathematics, not to itself:
closed-form impulse responses, steady-state sinusoid gain, linearity, zero
input, chunked == one-shot, dense solves of the banded system and of the
permuted block system of Eqs. 2-3, and scipy.signal.sosfilt as an
independent library routine.  tests/test_golden_paper_filters.py runs it on
the paper's benchmark designs and reproduces what Sec. IV-F reports about
their float32 realisations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sosfilt_oracle.c")
_SRC_WAVE = os.path.join(_HERE, "sosfilt_wavefront.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (-O2, no fast-math) into an in-tree shared library."""
    srcs = [_SRC, _SRC_WAVE]
    if not force and os.path.exists(_LIB_PATH) and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f)
                                                        for f in srcs):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, *srcs], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            for name in ("oracle_sosfilt_f32", "oracle_sosfilt_f64"):
                fn = getattr(lib, name)
                fn.argtypes = [ctypes.c_int, vp, vp, i64, vp, vp, vp]
                fn.restype = ctypes.c_int
            lib.oracle_sosfilt_batch_f32.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
            lib.oracle_sosfilt_batch_f32.restype = ctypes.c_int
            lib.oracle_sosfilt_wavefront_f32.argtypes = [ctypes.c_int, vp, vp, i64, vp, vp, vp, i64, ctypes.c_int]
            lib.oracle_sosfilt_wavefront_f32.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def sosfilt(sos, x, zi=None, return_state: bool = False, keep_output: bool = True):
    """Filter x (float32 or float64, 1-D) through the cascade ``sos`` [K][5] in float64.

    Returns y (float64) and, if ``return_state``, the final state zf [K][2].  With
    ``keep_output=False`` no output array is written (y is None): for timing runs.
    """
    lib = _load()
    sos = np.ascontiguousarray(np.asarray(sos, dtype=np.float64).reshape(-1, 5))
    k = sos.shape[0]
    x = np.ascontiguousarray(x)
    if x.dtype not in (np.float32, np.float64):
        x = x.astype(np.float64)
    n = x.shape[0]
    y = np.empty(n, dtype=np.float64) if keep_output else None
    zf = np.empty((k, 2), dtype=np.float64)
    zi_arr = None if zi is None else np.ascontiguousarray(np.asarray(zi, dtype=np.float64).reshape(k, 2))
    fn = lib.oracle_sosfilt_f32 if x.dtype == np.float32 else lib.oracle_sosfilt_f64
    rc = fn(k, _ptr(sos), _ptr(x), n, _ptr(zi_arr), _ptr(y), _ptr(zf))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return (y, zf) if return_state else y


def sosfilt_batch(sos_list, x_list, threads: int = 1, want_y: bool = True):
    """Independent signals (zero initial state), spread over ``threads`` host threads.

    Returns (list of y float64 arrays or None, list of zf arrays).
    """
    lib = _load()
    ks = np.array([np.asarray(s).reshape(-1, 5).shape[0] for s in sos_list], dtype=np.int32)
    sos_off = np.zeros(len(ks), dtype=np.int64)
    sos_off[1:] = np.cumsum(ks[:-1])
    sos_all = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.float64).reshape(-1, 5)
                                                   for s in sos_list]))
    ns = np.array([len(x) for x in x_list], dtype=np.int64)
    x_off = np.zeros(len(ns), dtype=np.int64)
    x_off[1:] = np.cumsum(ns[:-1])
    x_all = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float32) for x in x_list]))
    y_all = np.empty(x_all.shape[0], dtype=np.float64) if want_y else None
    zf_all = np.empty((int(ks.sum()), 2), dtype=np.float64)
    rc = lib.oracle_sosfilt_batch_f32(len(ks), _ptr(ks), _ptr(sos_off), _ptr(sos_all), _ptr(x_off), _ptr(ns),
                                      _ptr(x_all), _ptr(y_all), _ptr(zf_all), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    ys = [y_all[o:o + n] for o, n in zip(x_off, ns)] if want_y else None
    zfs = [zf_all[o:o + k] for o, k in zip(sos_off, ks)]
    return ys, zfs


def sosfilt_wavefront(sos, x, zi=None, return_state: bool = False, threads: int = 1, block: int = 4096,
                      keep_output: bool = True):
    """The same filtering as ``sosfilt`` for float32 x, run as the multi-core wavefront of Sec. III-A
    (groups of ``block`` samples carried through the sections by ``threads`` host threads).  Output
    and final state are bit-identical to ``sosfilt``'s."""
    lib = _load()
    sos = np.ascontiguousarray(np.asarray(sos, dtype=np.float64).reshape(-1, 5))
    k = sos.shape[0]
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    n = x.shape[0]
    y = np.empty(n, dtype=np.float64) if keep_output else None
    zf = np.empty((k, 2), dtype=np.float64)
    zi_arr = None if zi is None else np.ascontiguousarray(np.asarray(zi, dtype=np.float64).reshape(k, 2))
    rc = lib.oracle_sosfilt_wavefront_f32(k, _ptr(sos), _ptr(x), n, _ptr(zi_arr), _ptr(y), _ptr(zf), int(block),
                                          int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments or ran out of memory (code {rc})")
    return (y, zf) if return_state else y


def rel_err(y, y_ref) -> float:
    """The accuracy measure of Sec. IV-F: max |y - y_ref| / max |y_ref|."""
    y_ref = np.asarray(y_ref, dtype=np.float64)
    peak = float(np.max(np.abs(y_ref))) if y_ref.size else 0.0
    if y_ref.size == 0:
        return 0.0
    diff = float(np.max(np.abs(np.asarray(y, dtype=np.float64) - y_ref)))
    return diff / peak if peak > 0 else diff
