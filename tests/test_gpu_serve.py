"""GPU tests of the serving loop (sos_server_*): continuous batching over many streams with the
cascade state resident on the device between chunks.

Every stream's output over its chunks must equal one oracle run over the concatenated input (the
state is carried from chunk to chunk on the device), whether the stream is served alone or among
many others whose chunks arrive interleaved and are batched together, with a memory budget small
enough that requests queue.
"""
import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

from ._tol import bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    from paper_2607_23763_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _streams(n_streams, seed):
    out = []
    for s in range(n_streams):
        sos = workloads.serving_stream(seed + s)
        lens = [workloads.serving_chunk_len(seed + s, c, lo=1, hi=70000) for c in range(4)]
        chunks = [workloads.serving_chunk(seed + s, c, n) for c, n in enumerate(lens)]
        out.append((sos, chunks))
    return out


def _serve(streams, dev, budget, interleave=True):
    """Submit all chunks (round-robin over streams when interleaved), wait, return outputs per stream."""
    from paper_2607_23763_gb300 import SosServer
    srv = SosServer(budget_bytes=budget, max_batch=64, max_inflight=3)
    sids = [srv.add_stream(sos) for sos, _ in streams]
    rids = [[] for _ in streams]
    order = []
    n_chunks = max(len(c) for _, c in streams)
    if interleave:
        for c in range(n_chunks):
            for i, (_, chunks) in enumerate(streams):
                if c < len(chunks):
                    order.append((i, c))
    else:
        for i, (_, chunks) in enumerate(streams):
            order.extend((i, c) for c in range(len(chunks)))
    for i, c in order:
        x = torch.from_numpy(streams[i][1][c]).to(dev)
        rids[i].append(srv.submit(sids[i], x))
    srv.drain()
    comps = []
    while True:
        got = srv.poll(4096)
        if not got:
            break
        comps.extend(got)
    assert len(comps) == len(order)
    assert all(c["status"] == 0 for c in comps)
    outs = [torch.cat([srv.output(r) for r in rs]).cpu().numpy() for rs in rids]
    states = [srv.stream_state(sid, sos.shape[0]) for sid, (sos, _) in zip(sids, streams)]
    stats = srv.stats()
    srv.close()
    return outs, states, comps, stats


def test_serving_alone_and_in_mix_match_oracle(dev):
    streams = _streams(40, 700)
    mix_out, mix_states, comps, stats = _serve(streams, dev, budget=4 << 20)
    assert stats["completed"] == sum(len(c) for _, c in streams)
    assert stats["batches"] > 1  # the budget forced several batches
    for i, (sos, chunks) in enumerate(streams):
        x = np.concatenate(chunks)
        y_ref, zf_ref = oracle.sosfilt(sos, x, return_state=True)
        tol = bound(sos, x, y_ref, random_mix=True)
        err = oracle.rel_err(mix_out[i], y_ref)
        zerr = np.abs(mix_states[i] - zf_ref).max() / max(1e-30, np.abs(zf_ref).max())
        print(f"stream {i} K={sos.shape[0]} n={len(x)}: output error {err:.3e}, final-state error {zerr:.3e}, "
              f"bound {tol:.3e}")
        assert err < tol, i
        assert zerr < tol, i
        if i < 6:
            # the same stream served alone: the same chunks through the same batch kernel, each
            # continuing from the resident state, so the same output and state bit for bit
            alone, alone_states, _, _ = _serve([(sos, chunks)], dev, budget=4 << 20, interleave=False)
            assert np.array_equal(alone[0], mix_out[i]), i
            assert np.array_equal(alone_states[0], mix_states[i]), i


def test_serving_budget_queues_and_rejects(dev):
    from paper_2607_23763_gb300 import SosServer, SosError
    srv = SosServer(budget_bytes=1 << 20, max_batch=8, max_inflight=2)
    sid = srv.add_stream(designs.butter_lowpass(8, 0.1))
    big = torch.zeros((1 << 20) // 8 + 1, device=dev)
    with pytest.raises(SosError):
        srv.submit(sid, big)
    assert srv.stats()["rejected"] == 1
    # many chunks that fit one or two at a time: they queue and all complete, in order
    xs = [torch.from_numpy(workloads.normal_f32(9, 40000, stream=c)).to(dev) for c in range(12)]
    rids = [srv.submit(sid, x) for x in xs]
    srv.drain()
    y = torch.cat([srv.output(r) for r in rids]).cpu().numpy()
    x = np.concatenate([t.cpu().numpy() for t in xs])
    sos = designs.butter_lowpass(8, 0.1)
    assert oracle.rel_err(y, oracle.sosfilt(sos, x)) < 1e-4
    st = srv.stats()
    assert st["completed"] == 12 and st["inflight_bytes"] == 0
    srv.close()


def test_serving_replay_latencies(dev):
    """Replay with Poisson arrivals: every request completes, latencies are positive, results right."""
    from paper_2607_23763_gb300 import SosServer
    n_streams, per = 64, 6
    srv = SosServer(budget_bytes=64 << 20)
    soss = [workloads.serving_stream(900 + s) for s in range(n_streams)]
    sids = [srv.add_stream(sos) for sos in soss]
    rng = np.random.default_rng(1)
    lens = [[workloads.serving_chunk_len(900 + s, c) for c in range(per)] for s in range(n_streams)]
    xs = [[torch.from_numpy(workloads.serving_chunk(900 + s, c, lens[s][c])).to(dev) for c in range(per)]
          for s in range(n_streams)]
    ys = [[torch.empty_like(x) for x in row] for row in xs]
    order = [(s, c) for c in range(per) for s in range(n_streams)]
    t = np.cumsum(rng.exponential(20e-6, len(order)))
    lat = srv.replay([sids[s] for s, _ in order], [xs[s][c].data_ptr() for s, c in order],
                     [ys[s][c].data_ptr() for s, c in order], [lens[s][c] for s, c in order], t)
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    for s in range(0, n_streams, 8):
        x = np.concatenate([v.cpu().numpy() for v in xs[s]])
        y = np.concatenate([v.cpu().numpy() for v in ys[s]])
        y_ref = oracle.sosfilt(soss[s], x)
        assert oracle.rel_err(y, y_ref) < bound(soss[s], x, y_ref, random_mix=True), s
    srv.close()
