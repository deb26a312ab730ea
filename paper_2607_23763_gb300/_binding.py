"""ctypes binding of libsosfilt.so: argument marshalling only.

Every step of the filtering runs in the library's CUDA kernels; this module
only turns torch tensors into device pointers and the current torch stream
into a cudaStream_t.  There is no CPU fallback: if the library has not been
built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsosfilt.so")

SOS_OK, SOS_EINVAL, SOS_ENOMEM, SOS_ECUDA, SOS_ETIMEOUT, SOS_EUNSTABLE, SOS_EBUDGET = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "SOS_OK", -1: "SOS_EINVAL", -2: "SOS_ENOMEM", -3: "SOS_ECUDA", -4: "SOS_ETIMEOUT",
                -5: "SOS_EUNSTABLE", -6: "SOS_EBUDGET"}

# every symbol declared in include/sosfilt.h
EXPORTED = (
    "sos_filter_create", "sos_filter_destroy", "sos_filter_run", "sos_filter_run_batch",
    "sos_filter_stream_push", "sos_filter_stream_state", "sos_filter_sync_status", "sos_filter_trace",
    "sos_filter_run_host", "sos_filter_run_noalloc", "sos_filter_run_batch_ex", "sos_batch_sync_status",
    "sos_server_create", "sos_server_destroy", "sos_server_add_stream", "sos_server_submit", "sos_server_poll",
    "sos_server_drain", "sos_server_stream_state", "sos_server_get_stats", "sos_server_replay",
    "sos_autotune", "sos_autotune_choice", "sos_autotune_choice_ex", "sos_autotune_batch", "sos_autotune_batch_choice",
    "sos_batch_plan_create", "sos_batch_plan_launch",
    "sos_batch_plan_status", "sos_batch_plan_destroy", "sos_status_string",
)


class SosError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")


class Tuning(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_int), ("groups_per_cta", ctypes.c_int),
                ("threads_per_group", ctypes.c_int), ("fp64_carry", ctypes.c_int),
                ("spin_budget_cycles", ctypes.c_longlong), ("lookback_width", ctypes.c_int),
                ("carry", ctypes.c_int), ("solver", ctypes.c_int), ("deterministic", ctypes.c_int)]


CARRY_DEFAULT, CARRY_CASCADE, CARRY_SECTION = 0, 1, 2
HOST_DIRECT = -1  # sos_filter_run_host: the kernels read and write the pinned host buffers in place
SOLVER_DEFAULT, SOLVER_CR, SOLVER_PH, SOLVER_DTCR, SOLVER_TC = 0, 1, 2, 3, 4


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libsosfilt.so (built by ``paper_2607_23763_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.sos_filter_create.argtypes = [c_int, vp, vp, vp, ctypes.POINTER(vp)]
        lib.sos_filter_destroy.argtypes = [vp]
        lib.sos_filter_run.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.sos_filter_run_batch.argtypes = [c_int, vp, vp, vp, vp, vp]
        lib.sos_filter_run_batch_ex.argtypes = [c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.sos_batch_sync_status.argtypes = [c_int]
        lib.sos_server_create.argtypes = [vp, ctypes.POINTER(vp)]
        lib.sos_server_destroy.argtypes = [vp]
        lib.sos_server_add_stream.argtypes = [vp, c_int, vp, vp, ctypes.POINTER(c_int)]
        lib.sos_server_submit.argtypes = [vp, c_int, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
        lib.sos_server_poll.argtypes = [vp, vp, c_int, ctypes.POINTER(c_int), c_int]
        lib.sos_server_drain.argtypes = [vp]
        lib.sos_server_stream_state.argtypes = [vp, c_int, vp]
        lib.sos_server_get_stats.argtypes = [vp, vp]
        lib.sos_server_replay.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        lib.sos_autotune.argtypes = [c_int, vp]
        lib.sos_autotune_batch.argtypes = [vp]
        lib.sos_autotune_batch_choice.argtypes = [c_int, i64, ctypes.POINTER(c_int)]
        lib.sos_batch_plan_create.argtypes = [c_int, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
        lib.sos_batch_plan_launch.argtypes = [vp, vp]
        lib.sos_batch_plan_status.argtypes = [vp]
        lib.sos_batch_plan_destroy.argtypes = [vp]
        lib.sos_autotune_choice.argtypes = [c_int, i64, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.sos_autotune_choice_ex.argtypes = [c_int, i64, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                               ctypes.POINTER(c_int)]
        lib.sos_filter_stream_push.argtypes = [vp, vp, vp, i64, vp]
        lib.sos_filter_stream_state.argtypes = [vp, vp, vp, c_int]
        lib.sos_filter_sync_status.argtypes = [vp]
        lib.sos_filter_trace.argtypes = [vp, vp, i64]
        lib.sos_filter_run_host.argtypes = [vp, vp, vp, i64, vp, vp, i64]
        lib.sos_filter_run_noalloc.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.sos_status_string.argtypes = [c_int]
        lib.sos_status_string.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name == "sos_status_string":
                continue
            getattr(lib, name).restype = c_int
        _lib = lib
    return _lib


def _check(code: int, what: str):
    if code != SOS_OK:
        raise SosError(code, what)


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dptr(t, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t.data_ptr()


class SosFilter:
    """A cascade of K second-order sections (Eq. 1) bound to the current CUDA device.

    ``sos`` is [K][5] (b0, b1, b2, a1, a2) float64; ``zi`` the initial resident state [K][2].
    """

    def __init__(self, sos, zi=None, tuning: dict | None = None):
        lib = load_library()
        sos = np.ascontiguousarray(np.asarray(sos, dtype=np.float64).reshape(-1, 5))
        self.K = int(sos.shape[0])
        self.sos = sos
        zi_arr = None if zi is None else np.ascontiguousarray(np.asarray(zi, dtype=np.float32).reshape(self.K, 2))
        t = None
        if tuning:
            t = Tuning(**{k: int(v) for k, v in tuning.items()})
        h = ctypes.c_void_p()
        _check(lib.sos_filter_create(self.K, sos.ctypes.data, None if zi_arr is None else zi_arr.ctypes.data,
                                     None if t is None else ctypes.addressof(t), ctypes.byref(h)),
               "sos_filter_create")
        self._h = h
        self._lib = lib

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sos_filter_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def run(self, x, y=None, zi=None, zf=None, stream=None):
        """y = cascade(x) on the device; x, y, zi, zf are float32 CUDA tensors (y may be x)."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        n = x.numel()
        _check(self._lib.sos_filter_run(self._h, _dptr(x, "x"), _dptr(y, "y"), n,
                                        None if zi is None else _dptr(zi, "zi"),
                                        None if zf is None else _dptr(zf, "zf"), _stream_handle(stream)),
               "sos_filter_run")
        return y

    def run_noalloc(self, x, y, zi=None, zf=None, stream=None):
        """Like run(), but allocates nothing on the device (scratch in the library's fixed array).

        y must be supplied; at most 2^28 samples per call; calls must not overlap on the GPU.
        """
        _check(self._lib.sos_filter_run_noalloc(self._h, _dptr(x, "x"), _dptr(y, "y"), x.numel(),
                                                None if zi is None else _dptr(zi, "zi"),
                                                None if zf is None else _dptr(zf, "zf"), _stream_handle(stream)),
               "sos_filter_run_noalloc")
        return y

    def run_host(self, x, y=None, zi=None, chunk: int = 0, return_state: bool = False):
        """Filter a signal in host memory (numpy float32 or pinned CPU tensor); returns y (same kind).

        Copies in, filters and copies out in overlapping chunks inside the library; with
        ``chunk=HOST_DIRECT`` (pinned tensors only) the kernels work on the host buffers directly.
        """
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
                raise TypeError("x must be a contiguous float32 CPU tensor")
            if y is None:
                y = torch.empty_like(x, pin_memory=x.is_pinned())
            xp, yp, n = x.data_ptr(), y.data_ptr(), x.numel()
        else:
            x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
            if y is None:
                y = np.empty_like(x)
            xp, yp, n = x.ctypes.data, y.ctypes.data, x.size
        zi_arr = None if zi is None else np.ascontiguousarray(np.asarray(zi, dtype=np.float32).reshape(self.K, 2))
        zf = np.empty((self.K, 2), dtype=np.float32) if return_state else None
        _check(self._lib.sos_filter_run_host(self._h, xp, yp, n, None if zi_arr is None else zi_arr.ctypes.data,
                                             None if zf is None else zf.ctypes.data, int(chunk)),
               "sos_filter_run_host")
        return (y, zf) if return_state else y

    def stream_push(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(self._lib.sos_filter_stream_push(self._h, _dptr(x, "x"), _dptr(y, "y"), x.numel(),
                                                _stream_handle(stream)), "sos_filter_stream_push")
        return y

    def get_state(self) -> np.ndarray:
        z = np.empty((self.K, 2), dtype=np.float32)
        _check(self._lib.sos_filter_stream_state(self._h, z.ctypes.data, None, 0), "sos_filter_stream_state")
        return z

    def set_state(self, z):
        z = np.ascontiguousarray(np.asarray(z, dtype=np.float32).reshape(self.K, 2))
        _check(self._lib.sos_filter_stream_state(self._h, None, z.ctypes.data, 0), "sos_filter_stream_state")

    def set_trace(self, buf=None):
        """Enable the per-block phase trace into a uint64 CUDA tensor of shape [blocks, 32] (None = off)."""
        import torch
        if buf is None:
            _check(self._lib.sos_filter_trace(self._h, None, 0), "sos_filter_trace")
            return
        if not (buf.is_cuda and buf.dtype == torch.int64 and buf.is_contiguous() and buf.dim() == 2
                and buf.shape[1] == 32):
            raise TypeError("trace buffer must be a contiguous int64 CUDA tensor of shape [blocks, 32]")
        _check(self._lib.sos_filter_trace(self._h, buf.data_ptr(), buf.shape[0]), "sos_filter_trace")

    def sync_status(self) -> int:
        return int(self._lib.sos_filter_sync_status(self._h))


def run_batch(filters, xs, ys=None, zis=None, zfs=None, stream=None):
    """Filter many signals (each with its own filter object) in one batched call.

    ``zis``/``zfs``: optional lists of float32 CUDA tensors [K][2] (entries may be None) for the initial
    and final states; without them every signal starts from zero state (sos_filter_run_batch).
    """
    import torch
    lib = load_library()
    n = len(xs)
    if ys is None:
        ys = [torch.empty_like(x) for x in xs]
    hf = (ctypes.c_void_p * n)(*[f.handle for f in filters])
    hx = (ctypes.c_void_p * n)(*[_dptr(x, "x") for x in xs])
    hy = (ctypes.c_void_p * n)(*[_dptr(y, "y") for y in ys])
    hn = (ctypes.c_int64 * n)(*[x.numel() for x in xs])
    if zis is None and zfs is None:
        _check(lib.sos_filter_run_batch(n, ctypes.addressof(hf), ctypes.addressof(hx), ctypes.addressof(hy),
                                        ctypes.addressof(hn), _stream_handle(stream)), "sos_filter_run_batch")
        return ys
    def ptrs(ts, name):
        if ts is None:
            return None
        return (ctypes.c_void_p * n)(*[None if t is None else _dptr(t, name) for t in ts])
    hzi, hzf = ptrs(zis, "zi"), ptrs(zfs, "zf")
    _check(lib.sos_filter_run_batch_ex(n, ctypes.addressof(hf), ctypes.addressof(hx), ctypes.addressof(hy),
                                       ctypes.addressof(hn), None if hzi is None else ctypes.addressof(hzi),
                                       None if hzf is None else ctypes.addressof(hzf), _stream_handle(stream)),
           "sos_filter_run_batch_ex")
    return ys


def batch_sync_status(device: int = 0) -> int:
    """Synchronize the device and return the sticky status of its batched runs."""
    return int(load_library().sos_batch_sync_status(int(device)))


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int), ("max_inflight", ctypes.c_int)]


class Completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("stream_id", ctypes.c_int), ("status", ctypes.c_int),
                ("n", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "rejected", "batches", "max_batch_seen",
                                             "samples_done", "inflight_bytes")]


class SosServer:
    """Serving loop with continuous batching (sos_server_* in include/sosfilt.h).

    Streams keep their cascade state on the device between chunks; chunks name device tensors that
    must stay alive until they complete.
    """

    def __init__(self, budget_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0):
        self._lib = load_library()
        cfg = ServerConfig(int(budget_bytes), int(max_batch), int(max_inflight))
        h = ctypes.c_void_p()
        _check(self._lib.sos_server_create(ctypes.addressof(cfg), ctypes.byref(h)), "sos_server_create")
        self._h = h
        self._keep = {}  # request id -> tensors kept alive until completion

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sos_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def add_stream(self, sos, zi=None) -> int:
        sos = np.ascontiguousarray(np.asarray(sos, dtype=np.float64).reshape(-1, 5))
        K = sos.shape[0]
        zi_arr = None if zi is None else np.ascontiguousarray(np.asarray(zi, dtype=np.float32).reshape(K, 2))
        sid = ctypes.c_int()
        _check(self._lib.sos_server_add_stream(self._h, K, sos.ctypes.data,
                                               None if zi_arr is None else zi_arr.ctypes.data, ctypes.byref(sid)),
               "sos_server_add_stream")
        return sid.value

    def submit(self, stream_id: int, x, y=None) -> int:
        import torch
        if y is None:
            y = torch.empty_like(x)
        rid = ctypes.c_uint64()
        _check(self._lib.sos_server_submit(self._h, int(stream_id), _dptr(x, "x"), _dptr(y, "y"), x.numel(),
                                           ctypes.byref(rid)), "sos_server_submit")
        self._keep[rid.value] = (x, y)
        return rid.value

    def output(self, request_id: int):
        return self._keep[request_id][1]

    def poll(self, max_n: int = 1024, wait_ms: int = 0):
        """Completed requests as dicts (request_id, stream_id, status, n, t_submit, t_start, t_done)."""
        buf = (Completion * max_n)()
        n = ctypes.c_int()
        _check(self._lib.sos_server_poll(self._h, ctypes.addressof(buf), max_n, ctypes.byref(n), int(wait_ms)),
               "sos_server_poll")
        return [{f: getattr(buf[i], f) for f, _ in Completion._fields_} for i in range(n.value)]

    def drain(self):
        _check(self._lib.sos_server_drain(self._h), "sos_server_drain")

    def stream_state(self, stream_id: int, K: int) -> np.ndarray:
        z = np.empty((K, 2), dtype=np.float32)
        _check(self._lib.sos_server_stream_state(self._h, int(stream_id), z.ctypes.data), "sos_server_stream_state")
        return z

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.sos_server_get_stats(self._h, ctypes.addressof(st)), "sos_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def replay(self, stream_ids, x_ptrs, y_ptrs, lengths, t_arrival):
        """Replay requests at the given arrival offsets (seconds); returns per-request latency (s).

        x_ptrs / y_ptrs are integer device addresses (the caller keeps the memory alive).
        """
        m = len(stream_ids)
        sid = np.ascontiguousarray(np.asarray(stream_ids, dtype=np.int32))
        xp = np.ascontiguousarray(np.asarray(x_ptrs, dtype=np.uint64))
        yp = np.ascontiguousarray(np.asarray(y_ptrs, dtype=np.uint64))
        ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
        ta = np.ascontiguousarray(np.asarray(t_arrival, dtype=np.float64))
        lat = np.empty(m, dtype=np.float64)
        _check(self._lib.sos_server_replay(self._h, m, sid.ctypes.data, xp.ctypes.data, yp.ctypes.data,
                                           ln.ctypes.data, ta.ctypes.data, lat.ctypes.data), "sos_server_replay")
        return lat


def autotune(max_log2n: int = 0) -> np.ndarray:
    """Time the candidate launch configurations on the current device and keep the fastest per
    (section count, length); returns the measured GS/s as [8 sections][4 lengths][CR32, CR64, PH, DTCR,
    PH with 10 groups per tile, PH on the tensor cores]."""
    rep = np.zeros((8, 4, 6), dtype=np.float32)
    _check(load_library().sos_autotune(int(max_log2n), rep.ctypes.data), "sos_autotune")
    return rep


def autotune_choice(n_sections: int, n: int, with_groups: bool = False):
    """(solver, N) the autotuner picked for this section count and length; (0, 0) if none.  With
    with_groups, (solver, N, groups per tile)."""
    s, N, W = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().sos_autotune_choice_ex(int(n_sections), int(n), ctypes.byref(s), ctypes.byref(N),
                                                 ctypes.byref(W)), "sos_autotune_choice_ex")
    return (s.value, N.value, W.value) if with_groups else (s.value, N.value)


def autotune_batch() -> np.ndarray:
    """Time the batch kernel's tile geometries (N = 64, N = 32) on the current device and keep the
    faster per (section count, signal length); returns the measured GS/s as [8 sections][signal
    lengths 2^12, 2^15, 2^18, 2^21][N = 64, N = 32]."""
    rep = np.zeros((8, 4, 2), dtype=np.float32)
    _check(load_library().sos_autotune_batch(rep.ctypes.data), "sos_autotune_batch")
    return rep


def autotune_batch_choice(n_sections: int, n: int) -> int:
    """Samples per thread the batch autotuner picked for this section count and signal length; 0 if
    it has not run."""
    N = ctypes.c_int()
    _check(load_library().sos_autotune_batch_choice(int(n_sections), int(n), ctypes.byref(N)),
           "sos_autotune_batch_choice")
    return N.value


class BatchPlan:
    """A prepared batch (sos_batch_plan_*): launch() enqueues it with no host-side work, so it can be
    captured into a CUDA graph (torch.cuda.graph) and replayed.  Keeps its tensors and filters alive."""

    def __init__(self, filters, xs, ys=None, zis=None, zfs=None):
        import torch
        self._lib = load_library()
        n = len(xs)
        if ys is None:
            ys = [torch.empty_like(x) for x in xs]
        self.filters, self.xs, self.ys, self.zis, self.zfs = list(filters), list(xs), list(ys), zis, zfs
        hf = (ctypes.c_void_p * n)(*[f.handle for f in filters])
        hx = (ctypes.c_void_p * n)(*[_dptr(x, "x") for x in xs])
        hy = (ctypes.c_void_p * n)(*[_dptr(y, "y") for y in ys])
        hn = (ctypes.c_int64 * n)(*[x.numel() for x in xs])
        def ptrs(ts, name):
            return None if ts is None else (ctypes.c_void_p * n)(*[None if t is None else _dptr(t, name) for t in ts])
        hzi, hzf = ptrs(zis, "zi"), ptrs(zfs, "zf")
        h = ctypes.c_void_p()
        _check(self._lib.sos_batch_plan_create(n, ctypes.addressof(hf), ctypes.addressof(hx), ctypes.addressof(hy),
                                               ctypes.addressof(hn), None if hzi is None else ctypes.addressof(hzi),
                                               None if hzf is None else ctypes.addressof(hzf), ctypes.byref(h)),
               "sos_batch_plan_create")
        self._h = h

    def launch(self, stream=None):
        _check(self._lib.sos_batch_plan_launch(self._h, _stream_handle(stream)), "sos_batch_plan_launch")
        return self.ys

    def status(self) -> int:
        return int(self._lib.sos_batch_plan_status(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sos_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
