"""The serving loop's host logic on the CPU: sosfilt_server.cpp compiled against host stand-ins for
the CUDA runtime and for the library's filters and batched run (tests/server_host/).

A stream of the stand-in runtime is a worker thread that runs its work in order; the stand-in
batched run filters in float64 and keeps float32 states between chunks, as the library does, and
records how many batches and bytes were in flight at once.  The tests check admission by the
memory budget, one chunk in flight per stream and the chunks of a stream in order, batches that
overlap, rejection of chunks larger than the budget, the up-front checks of a replay, the resident
state, a failed batch reported on its requests and as the server's sticky status, and that
destroying the server finishes its queued work.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads
from paper_2607_23763_gb300._binding import Completion, ServerConfig, ServerStats
from workloads import designs

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRCS = [os.path.join(_HERE, "server_host", "server_host.cpp"),
         os.path.join(_ROOT, "paper_2607_23763_gb300", "csrc", "sosfilt_server.cpp")]
_DEPS = _SRCS + [os.path.join(_HERE, "server_host", "cuda_runtime.h"), os.path.join(_ROOT, "include", "sosfilt.h")]
_LIB = os.path.join(_HERE, "_build", "libserver_host.so")
SOS_OK, SOS_EINVAL, SOS_EBUDGET = 0, -1, -6


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not os.path.exists(_LIB) or any(os.path.getmtime(d) > os.path.getmtime(_LIB) for d in _DEPS):
        tmp = f"{_LIB}.{os.getpid()}.tmp"  # parallel test workers build side by side
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread",
                        "-I", os.path.join(_HERE, "server_host"), "-I", os.path.join(_ROOT, "include"),
                        "-o", tmp, *_SRCS], check=True)
        os.replace(tmp, _LIB)
    L = ctypes.CDLL(_LIB)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sos_server_create.argtypes = [vp, ctypes.POINTER(vp)]
    L.sos_server_destroy.argtypes = [vp]
    L.sos_server_add_stream.argtypes = [vp, c_int, vp, vp, ctypes.POINTER(c_int)]
    L.sos_server_submit.argtypes = [vp, c_int, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
    L.sos_server_poll.argtypes = [vp, vp, c_int, ctypes.POINTER(c_int), c_int]
    L.sos_server_drain.argtypes = [vp]
    L.sos_server_stream_state.argtypes = [vp, c_int, vp]
    L.sos_server_get_stats.argtypes = [vp, vp]
    L.sos_server_replay.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.host_stats.argtypes = [vp]
    L.host_reset.argtypes = [c_int]
    L.host_fail_next.argtypes = [c_int]
    return L


class Server:
    def __init__(self, L, budget, max_batch=8, max_inflight=3, delay_us=300):
        self.L = L
        L.host_reset(delay_us)
        cfg = ServerConfig(budget, max_batch, max_inflight)
        self.h = ctypes.c_void_p()
        assert L.sos_server_create(ctypes.byref(cfg), ctypes.byref(self.h)) == SOS_OK
        self.keep = []

    def add(self, sos):
        sos = np.ascontiguousarray(sos, dtype=np.float64)
        sid = ctypes.c_int()
        assert self.L.sos_server_add_stream(self.h, sos.shape[0], sos.ctypes.data, None, ctypes.byref(sid)) == SOS_OK
        return sid.value

    def submit(self, sid, x, y):
        self.keep += [x, y]
        rid = ctypes.c_uint64()
        rc = self.L.sos_server_submit(self.h, sid, x.ctypes.data, y.ctypes.data, x.size, ctypes.byref(rid))
        return rc, rid.value

    def poll_all(self, n_expected):
        out = (Completion * 256)()
        got = []
        while len(got) < n_expected:
            k = ctypes.c_int()
            assert self.L.sos_server_poll(self.h, out, 256, ctypes.byref(k), 100) == SOS_OK
            got += [(c.request_id, c.stream_id, c.status, c.n, c.t_submit, c.t_start, c.t_done)
                    for c in out[:k.value]]
        return got

    def stats(self):
        st = ServerStats()
        assert self.L.sos_server_get_stats(self.h, ctypes.byref(st)) == SOS_OK
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def host(self):
        a = (ctypes.c_longlong * 3)()
        self.L.host_stats(a)
        return {"max_batches": a[0], "max_bytes": a[1], "batches": a[2]}

    def close(self):
        assert self.L.sos_server_destroy(self.h) == SOS_OK


def _streams(n_streams, per, seed):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_streams):
        order = [2, 4, 8, 16][s % 4]
        sos = designs.butter_lowpass(order, 0.2 if order < 16 else 0.05)
        lens = rng.integers(100, 3000, per)
        x = workloads.normal_f32(300 + s, int(lens.sum()))
        chunks = np.split(x, np.cumsum(lens)[:-1])
        out.append((sos, [np.ascontiguousarray(c) for c in chunks]))
    return out


def test_continuous_batching_keeps_each_stream_in_order_within_budget(lib):
    budget = 256 << 10
    srv = Server(lib, budget, delay_us=2000)  # batches long enough to overlap even on a loaded host
    streams = _streams(12, 6, 1)
    sids = [srv.add(sos) for sos, _ in streams]
    ys = [[np.full_like(c, np.nan) for c in chunks] for _, chunks in streams]
    rid_of = {}
    for c in range(6):  # chunks of different streams interleaved
        for s, (_, chunks) in enumerate(streams):
            rc, rid = srv.submit(sids[s], chunks[c], ys[s][c])
            assert rc == SOS_OK
            rid_of[rid] = (s, c)
    comps = srv.poll_all(12 * 6)
    st, host = srv.stats(), srv.host()
    srv.close()
    assert all(status == SOS_OK for _, _, status, *_ in comps)
    assert sorted(rid_of[r] for r, *_ in comps) == sorted(rid_of.values())
    # one chunk of a stream in flight at a time, the chunks of a stream in order
    by_stream = {}
    for rid, sid, status, n, t_sub, t_start, t_done in comps:
        s, c = rid_of[rid]
        by_stream.setdefault(s, []).append((c, t_start, t_done))
    for s, rows in by_stream.items():
        rows.sort()
        assert [c for c, _, _ in rows] == list(range(6))
        for (_, _, done), (_, start, _) in zip(rows, rows[1:]):
            assert start >= done, s
    # each stream's chunks continue from the resident state: the same as one long call
    for s, (sos, chunks) in enumerate(streams):
        y_ref = oracle.sosfilt(sos, np.concatenate(chunks))
        assert oracle.rel_err(np.concatenate(ys[s]), y_ref) < 1e-5, s
    assert st["submitted"] == st["completed"] == 72 and st["rejected"] == 0
    assert 1 <= st["max_batch_seen"] <= 8
    # admission by the budget; batches overlapped
    assert host["max_bytes"] <= budget
    assert 2 <= host["max_batches"] <= 3


def test_a_chunk_larger_than_the_budget_is_rejected(lib):
    srv = Server(lib, budget=8 << 10)
    sid = srv.add(designs.butter_lowpass(4, 0.2))
    x = workloads.normal_f32(7, 2048)  # 16 KiB in and out
    rc, _ = srv.submit(sid, x, np.empty_like(x))
    assert rc == SOS_EBUDGET
    small = np.ascontiguousarray(x[:512])
    y = np.empty_like(small)
    rc, _ = srv.submit(sid, small, y)
    assert rc == SOS_OK
    srv.poll_all(1)
    st = srv.stats()
    srv.close()
    assert st["rejected"] == 1 and st["completed"] == 1
    assert oracle.rel_err(y, oracle.sosfilt(designs.butter_lowpass(4, 0.2), small)) < 1e-5


def _replay(srv, sids, xs, ys, t):
    m = len(sids)
    sid = np.ascontiguousarray(sids, dtype=np.int32)
    xp = np.array([a.ctypes.data for a in xs], dtype=np.uint64)
    yp = np.array([a.ctypes.data for a in ys], dtype=np.uint64)
    n = np.array([a.size for a in xs], dtype=np.int64)
    ta = np.ascontiguousarray(t, dtype=np.float64)
    lat = np.zeros(m)
    rc = srv.L.sos_server_replay(srv.h, m, sid.ctypes.data, xp.ctypes.data, yp.ctypes.data, n.ctypes.data,
                                 ta.ctypes.data, lat.ctypes.data)
    return rc, lat


def test_replay_checks_every_request_before_queueing_any(lib):
    srv = Server(lib, budget=64 << 10, delay_us=100)
    sos = designs.butter_lowpass(8, 0.2)
    sids = [srv.add(sos) for _ in range(4)]
    xs = [workloads.normal_f32(20 + i, 1000) for i in range(8)]
    ys = [np.full_like(x, np.nan) for x in xs]
    order = [sids[i % 4] for i in range(8)]
    t = np.arange(8) * 1e-4
    big = workloads.normal_f32(30, 9000)  # 72 KB: over the budget
    rc, _ = _replay(srv, order[:3] + [sids[0]], xs[:3] + [big], ys[:3] + [np.empty_like(big)], t[:4])
    assert rc == SOS_EBUDGET
    rc, _ = _replay(srv, order[:2] + [99], xs[:3], ys[:3], t[:3])
    assert rc == SOS_EINVAL
    assert srv.stats()["submitted"] == 0  # nothing of either was queued
    assert all(np.isnan(y).all() for y in ys)
    rc, lat = _replay(srv, order, xs, ys, t)
    st = srv.stats()
    srv.close()
    assert rc == SOS_OK and np.all(lat > 0) and st["completed"] == 8
    for s in range(4):
        mine = [i for i in range(8) if i % 4 == s]
        y_ref = oracle.sosfilt(sos, np.concatenate([xs[i] for i in mine]))
        assert oracle.rel_err(np.concatenate([ys[i] for i in mine]), y_ref) < 1e-5


def test_resident_state_after_the_chunks(lib):
    srv = Server(lib, budget=1 << 20)
    sos = designs.butter_lowpass(6, 0.2)
    sid = srv.add(sos)
    chunks = [workloads.normal_f32(40 + i, 700 + 100 * i) for i in range(5)]
    for c in chunks:
        assert srv.submit(sid, c, np.empty_like(c))[0] == SOS_OK
    z = np.zeros((3, 2), dtype=np.float32)
    assert lib.sos_server_stream_state(srv.h, sid, z.ctypes.data) == SOS_OK  # waits for the chunks
    srv.close()
    _, zf = oracle.sosfilt(sos, np.concatenate(chunks), return_state=True)
    assert np.abs(z - zf).max() <= 1e-5 * max(1.0, np.abs(zf).max())


def test_destroy_finishes_the_queued_work(lib):
    srv = Server(lib, budget=32 << 10, max_inflight=2, delay_us=500)
    sos = designs.butter_lowpass(2, 0.2)
    sids = [srv.add(sos) for _ in range(3)]
    xs = [workloads.normal_f32(60 + i, 1500) for i in range(12)]
    ys = [np.full_like(x, np.nan) for x in xs]
    for i, (x, y) in enumerate(zip(xs, ys)):
        assert srv.submit(sids[i % 3], x, y)[0] == SOS_OK
    srv.close()  # returns once every queued chunk has run
    assert all(np.isfinite(y).all() for y in ys)


def test_a_failed_batch_is_reported_and_its_streams_keep_their_state(lib):
    SOS_ECUDA = -3
    srv = Server(lib, budget=1 << 20, max_batch=4, max_inflight=1, delay_us=100)
    sos = designs.butter_lowpass(4, 0.2)
    sids = [srv.add(sos) for _ in range(2)]
    lib.host_fail_next(1)  # the first batch is refused
    xs = [workloads.normal_f32(80 + i, 600) for i in range(6)]
    ys = [np.full_like(x, np.nan) for x in xs]
    rid_of = {}
    for i in range(6):
        rc, rid = srv.submit(sids[i % 2], xs[i], ys[i])
        assert rc == SOS_OK
        rid_of[rid] = i
    out = (Completion * 16)()
    status = {}
    while len(status) < 6:
        k = ctypes.c_int()
        rc = lib.sos_server_poll(srv.h, out, 16, ctypes.byref(k), 100)
        status.update({rid_of[c.request_id]: c.status for c in out[:k.value]})
    assert rc == SOS_ECUDA  # the first error of any batch, sticky
    assert lib.sos_server_drain(srv.h) == SOS_ECUDA
    failed = sorted(i for i, st in status.items() if st != SOS_OK)
    assert failed and all(status[i] == SOS_ECUDA for i in failed)
    assert all(i < 4 for i in failed)  # the first batch held at most the first chunk of each stream
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["inflight_bytes"] == 0
    # each stream continues from its state before the failed chunk, as if that chunk were skipped
    for s in range(2):
        z = np.zeros((2, 2))
        for i in range(s, 6, 2):
            if i in failed:
                assert np.isnan(ys[i]).all()
                continue
            y_ref, z = oracle.sosfilt(sos, xs[i], zi=z, return_state=True)
            assert oracle.rel_err(ys[i], y_ref) < 1e-5, i
