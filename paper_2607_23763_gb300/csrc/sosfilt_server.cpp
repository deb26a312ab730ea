// Serving loop: continuous batching of filtering requests from many streams, each stream's
// cascade state resident on the device between chunks (declared in include/sosfilt.h).
//
// A stream is a cascade (its own sos_filter) plus two device copies of its [K][2] state; a batch
// reads one copy and writes the other, and the stream's current copy flips when its chunk is
// admitted, so chunk i + 1 continues from chunk i's final state without a host round trip.
// Requests name caller-owned device buffers.  A scheduler thread admits the oldest ready chunks
// (streams with a queued chunk and none in flight) while the bytes in flight stay inside the
// memory budget; two launcher threads issue the admitted batches through sos_filter_run_batch_ex on
// a few CUDA streams, so that several batches overlap on the device and admission, planning and
// issuing overlap; a host function behind every batch hands it to a completion thread, which
// releases its streams and budget.  New requests are admitted as soon as budget and batch slots
// free up.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sosfilt.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Req {
    uint64_t id = 0;
    int sid = 0;
    const float *x = nullptr;
    float *y = nullptr;
    int64_t n = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = SOS_OK;
    // fixed at admission: the stream's filter and the state copies this chunk reads and writes
    sos_filter *f = nullptr;
    const float *zi = nullptr;
    float *zf = nullptr;
};

struct Stream {
    sos_filter *f = nullptr;
    int K = 0;
    float *d_state[2] = {nullptr, nullptr};
    int cur = 0;
    std::deque<Req> q;  // queued chunks, in submission order
    bool busy = false;  // a chunk in flight
};

struct Batch;

}  // namespace

struct sos_server {
    int device = 0;
    sos_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv;     // scheduler: new work or completions
    std::condition_variable cv_done;  // drain and state readers: streams released
    std::deque<Stream> streams;     // a deque: adding a stream never moves the others
    std::deque<int> ready;          // idle streams with a queued chunk, in order of readiness
    // completion records for the pollers, under their own lock, so that collecting them does not
    // hold up admission
    std::mutex mu_rec;
    std::condition_variable cv_rec;
    std::vector<sos_completion> done;
    uint64_t next_id = 1;
    int64_t inflight_bytes = 0;
    int inflight_batches = 0;
    int64_t queued = 0;             // requests submitted and not yet completed
    sos_server_stats stats{};
    std::vector<cudaStream_t> cstreams;
    int next_cs = 0;
    bool stop = false;
    std::atomic<int> sticky{SOS_OK};  // first error of a batch launch (written under mu)
    std::deque<Batch *> to_launch;  // admitted batches, in admission order, for the launcher threads
    std::condition_variable cv_launch;
    bool sched_done = false;        // the scheduler has exited; the launchers drain and exit
    // batches whose device work has finished, for the completion thread (their own lock: the CUDA
    // host function behind a batch only hands it over)
    std::mutex mu_fin;
    std::condition_variable cv_fin;
    std::deque<Batch *> finished;
    bool fin_stop = false;
    std::thread sched, launchers[2], completer;
};

namespace {

struct Batch {
    sos_server *srv = nullptr;
    std::vector<Req> reqs;
    int64_t bytes = 0;
    double t_done = 0;  // when its device work finished
};

int64_t req_bytes(const Req &r) { return (r.x == r.y ? 4 : 8) * r.n; }

constexpr double kFillWait = 200e-6;  // seconds a small batch may wait to fill while the device is busy

// Completion bookkeeping of a batch whose device work has finished (no CUDA calls): records for the
// pollers, the streams' next chunks made ready, the budget released.
void complete_batch(Batch *b) {
    sos_server *s = b->srv;
    const double t = b->t_done;
    // the completion records are built before the lock is taken; under it, one append and the
    // streams' bookkeeping
    std::vector<sos_completion> recs(b->reqs.size());
    int64_t samples = 0;
    for (size_t i = 0; i < b->reqs.size(); ++i) {
        const Req &r = b->reqs[i];
        recs[i] = sos_completion{r.id, r.sid, r.status, r.n, r.t_submit, r.t_start, t};
        samples += r.n;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Req &r : b->reqs) {
            Stream &st = s->streams[r.sid];
            st.busy = false;
            if (!st.q.empty()) s->ready.push_back(r.sid);
        }
        const int64_t m = static_cast<int64_t>(b->reqs.size());
        s->stats.completed += m;
        s->stats.samples_done += samples;
        s->queued -= m;
        s->inflight_bytes -= b->bytes;
        s->inflight_batches -= 1;
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
    {
        std::lock_guard<std::mutex> lk(s->mu_rec);
        s->done.insert(s->done.end(), recs.begin(), recs.end());
    }
    s->cv_rec.notify_all();
    delete b;
}

// Host function behind a batch on its CUDA stream: it stamps the completion time and hands the
// batch to the completion thread, so that the CUDA stream's next batch does not wait on the
// bookkeeping.
void CUDART_CB batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    sos_server *s = b->srv;
    b->t_done = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu_fin);
        s->finished.push_back(b);
    }
    s->cv_fin.notify_one();
}

void completer(sos_server *s) {
    std::unique_lock<std::mutex> lk(s->mu_fin);
    for (;;) {
        s->cv_fin.wait(lk, [&] { return !s->finished.empty() || s->fin_stop; });
        if (s->finished.empty()) break;  // stopping, and every batch has been completed
        Batch *b = s->finished.front();
        s->finished.pop_front();
        lk.unlock();
        complete_batch(b);
        lk.lock();
    }
}

// Admission: the oldest ready chunks while the budget allows, with each chunk's filter and state
// copies fixed here (a stream's current copy flips per admitted chunk); the batch then goes to the
// launcher thread, so that admitting the next batch overlaps with issuing this one.
void scheduler(sos_server *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    double fill_since = 0;  // when a small batch started waiting to fill
    for (;;) {
        if (s->stop && s->queued == 0) break;
        Batch *b = nullptr;
        // while two or more batches keep the device busy, a batch waits up to kFillWait to gather half
        // of the largest batch: fewer, larger batches cost less per chunk on the host (half measured
        // 13 % more capacity than a quarter)
        bool fill = false;
        if (s->inflight_batches >= 2 && static_cast<int64_t>(s->ready.size()) < s->cfg.max_batch / 2 && !s->stop) {
            const double t = now_s();
            if (fill_since == 0) fill_since = t;
            fill = t - fill_since < kFillWait;
        }
        if (!fill && s->inflight_batches < s->cfg.max_inflight && !s->ready.empty()) {
            fill_since = 0;
            b = new (std::nothrow) Batch();
            if (b) {
                b->srv = s;
                b->reqs.reserve(std::min<size_t>(s->ready.size(), static_cast<size_t>(s->cfg.max_batch)));
                const double t = now_s();
                while (!s->ready.empty() && static_cast<int>(b->reqs.size()) < s->cfg.max_batch) {
                    Stream &st = s->streams[s->ready.front()];
                    const int64_t need = req_bytes(st.q.front());
                    if (s->inflight_bytes + b->bytes + need > s->cfg.budget_bytes) break;  // oldest first
                    b->reqs.push_back(st.q.front());
                    Req &r = b->reqs.back();
                    st.q.pop_front();
                    st.busy = true;
                    r.t_start = t;
                    r.f = st.f;
                    r.zi = st.d_state[st.cur];
                    r.zf = st.d_state[st.cur ^ 1];
                    st.cur ^= 1;
                    b->bytes += need;
                    s->ready.pop_front();
                }
                if (b->reqs.empty()) {
                    delete b;
                    b = nullptr;
                } else {
                    s->inflight_bytes += b->bytes;
                    s->inflight_batches += 1;
                    s->stats.batches += 1;
                    s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, b->reqs.size());
                }
            }
        }
        if (!b) {
            if (fill)
                s->cv.wait_for(lk, std::chrono::microseconds(50));
            else
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        s->to_launch.push_back(b);
        s->cv_launch.notify_one();
    }
    s->sched_done = true;
    s->cv_launch.notify_all();
}

// Issue: one batched run per admitted batch, on the next of the server's CUDA streams, with a host
// function behind it for the completions.  Two launcher threads take batches in admission order and
// plan them at the same time (the library's batched runs plan concurrently on separate scratch);
// the streams of a batch's requests are busy, so nobody else touches their state copies meanwhile.
void launcher(sos_server *s) {
    if (cudaSetDevice(s->device) != cudaSuccess) return;
    std::vector<sos_filter *> fs;
    std::vector<const float *> xs, zis;
    std::vector<float *> ys, zfs;
    std::vector<int64_t> ns;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_launch.wait(lk, [&] { return !s->to_launch.empty() || s->sched_done; });
        if (s->to_launch.empty()) break;  // the scheduler has exited and nothing is left
        Batch *b = s->to_launch.front();
        s->to_launch.pop_front();
        cudaStream_t cs = s->cstreams[s->next_cs];
        s->next_cs = (s->next_cs + 1) % static_cast<int>(s->cstreams.size());
        lk.unlock();
        const size_t m = b->reqs.size();
        fs.resize(m);
        xs.resize(m);
        ys.resize(m);
        ns.resize(m);
        zis.resize(m);
        zfs.resize(m);
        for (size_t i = 0; i < m; ++i) {
            const Req &r = b->reqs[i];
            fs[i] = r.f;
            xs[i] = r.x;
            ys[i] = r.y;
            ns[i] = r.n;
            zis[i] = r.zi;
            zfs[i] = r.zf;
        }
        sos_status st = sos_filter_run_batch_ex(static_cast<int>(m), fs.data(), xs.data(), ys.data(), ns.data(),
                                                zis.data(), zfs.data(), cs);
        if (st != SOS_OK) {
            for (Req &r : b->reqs) r.status = st;
            // the batch did not run: its streams keep the state they had before it.  This happens
            // before the batch can complete, while its streams are still busy, so none of them can
            // have been admitted again meanwhile.
            lk.lock();
            if (s->sticky == SOS_OK) s->sticky = st;
            for (const Req &r : b->reqs) s->streams[r.sid].cur ^= 1;
            lk.unlock();
        }
        const bool queued_ok = cudaLaunchHostFunc(cs, batch_done, b) == cudaSuccess;
        lk.lock();
        if (!queued_ok) {  // complete it here so that pollers and the budget are not stuck
            if (s->sticky == SOS_OK) s->sticky = SOS_ECUDA;
            for (Req &r : b->reqs) r.status = SOS_ECUDA;
            lk.unlock();
            batch_done(b);
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

sos_status sos_server_create(const sos_server_config *cfg, sos_server **out) {
    if (!out) return SOS_EINVAL;
    *out = nullptr;
    sos_server *s = new (std::nothrow) sos_server();
    if (!s) return SOS_ENOMEM;
    if (cfg) s->cfg = *cfg;
    if (s->cfg.budget_bytes <= 0) s->cfg.budget_bytes = 16LL << 30;
    if (s->cfg.max_batch <= 0) s->cfg.max_batch = 4096;
    if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 4;
    if (s->cfg.max_inflight > 8) s->cfg.max_inflight = 8;  // the library keeps eight batch scratch sets
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return SOS_ECUDA;
    }
    s->cstreams.resize(s->cfg.max_inflight);
    for (auto &c : s->cstreams)
        if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return SOS_ECUDA;
        }
    auto stop_threads = [s] {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->sched_done = true;
        }
        s->cv_launch.notify_all();
        for (auto &l : s->launchers)
            if (l.joinable()) l.join();
        {
            std::lock_guard<std::mutex> lk(s->mu_fin);
            s->fin_stop = true;
        }
        s->cv_fin.notify_all();
        if (s->completer.joinable()) s->completer.join();
    };
    try {
        s->completer = std::thread(completer, s);
        for (auto &l : s->launchers) l = std::thread(launcher, s);
    } catch (...) {
        stop_threads();
        delete s;
        return SOS_ENOMEM;
    }
    try {
        s->sched = std::thread(scheduler, s);
    } catch (...) {
        stop_threads();
        delete s;
        return SOS_ENOMEM;
    }
    *out = s;
    return SOS_OK;
}

sos_status sos_server_destroy(sos_server *s) {
    if (!s) return SOS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();  // after every queued request has completed
    for (auto &l : s->launchers)
        if (l.joinable()) l.join();
    {
        std::lock_guard<std::mutex> lk(s->mu_fin);
        s->fin_stop = true;
    }
    s->cv_fin.notify_all();
    if (s->completer.joinable()) s->completer.join();
    cudaSetDevice(s->device);
    for (auto &c : s->cstreams) cudaStreamSynchronize(c);
    // the filters before the CUDA streams their last batches ran on
    for (auto &st : s->streams) {
        sos_filter_destroy(st.f);
        cudaFree(st.d_state[0]);
        cudaFree(st.d_state[1]);
    }
    for (auto &c : s->cstreams) cudaStreamDestroy(c);
    delete s;
    return SOS_OK;
}

sos_status sos_server_add_stream(sos_server *s, int n_sections, const double *sos, const float *zi, int *stream_id) {
    if (!s || !stream_id || n_sections < 1 || n_sections > 64 || !sos) return SOS_EINVAL;
    if (cudaSetDevice(s->device) != cudaSuccess) return SOS_ECUDA;
    Stream st;
    st.K = n_sections;
    sos_status rc = sos_filter_create(n_sections, sos, nullptr, nullptr, &st.f);
    if (rc != SOS_OK) return rc;
    const size_t bytes = sizeof(float) * 2 * n_sections;
    if (cudaMalloc(&st.d_state[0], bytes) != cudaSuccess || cudaMalloc(&st.d_state[1], bytes) != cudaSuccess) {
        cudaGetLastError();
        sos_filter_destroy(st.f);
        cudaFree(st.d_state[0]);
        return SOS_ENOMEM;
    }
    std::vector<float> z(2 * n_sections, 0.f);
    if (zi) std::memcpy(z.data(), zi, bytes);
    if (cudaMemcpy(st.d_state[0], z.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        sos_filter_destroy(st.f);
        cudaFree(st.d_state[0]);
        cudaFree(st.d_state[1]);
        return SOS_ECUDA;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->streams.push_back(std::move(st));
    *stream_id = static_cast<int>(s->streams.size()) - 1;
    return SOS_OK;
}

sos_status sos_server_submit(sos_server *s, int stream_id, const float *x_dev, float *y_dev, int64_t n,
                             uint64_t *request_id) {
    if (!s || n <= 0 || !x_dev || !y_dev) return SOS_EINVAL;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (stream_id < 0 || stream_id >= static_cast<int>(s->streams.size())) return SOS_EINVAL;
        Req r;
        r.id = s->next_id++;
        r.sid = stream_id;
        r.x = x_dev;
        r.y = y_dev;
        r.n = n;
        r.t_submit = t;
        if (req_bytes(r) > s->cfg.budget_bytes) {
            s->stats.rejected += 1;
            return SOS_EBUDGET;
        }
        Stream &st = s->streams[stream_id];
        if (!st.busy && st.q.empty()) s->ready.push_back(stream_id);
        st.q.push_back(r);
        s->queued += 1;
        s->stats.submitted += 1;
        if (request_id) *request_id = r.id;
    }
    s->cv.notify_one();
    return SOS_OK;
}

sos_status sos_server_poll(sos_server *s, sos_completion *out, int max, int *n_out, int wait_ms) {
    if (!s || !n_out || max < 0 || (max > 0 && !out)) return SOS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu_rec);
    if (s->done.empty() && wait_ms > 0)
        s->cv_rec.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    const int k = std::min<int>(max, static_cast<int>(s->done.size()));
    for (int i = 0; i < k; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n_out = k;
    return static_cast<sos_status>(s->sticky.load());
}

sos_status sos_server_drain(sos_server *s) {
    if (!s) return SOS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->queued == 0; });
    return static_cast<sos_status>(s->sticky.load());
}

sos_status sos_server_stream_state(sos_server *s, int stream_id, float *z_host) {
    if (!s || !z_host) return SOS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (stream_id < 0 || stream_id >= static_cast<int>(s->streams.size())) return SOS_EINVAL;
    s->cv_done.wait(lk, [&] {
        const Stream &st = s->streams[stream_id];
        return !st.busy && st.q.empty();
    });
    const Stream &st = s->streams[stream_id];
    if (cudaSetDevice(s->device) != cudaSuccess) return SOS_ECUDA;
    if (cudaMemcpy(z_host, st.d_state[st.cur], sizeof(float) * 2 * st.K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOS_ECUDA;
    return SOS_OK;
}

sos_status sos_server_get_stats(sos_server *s, sos_server_stats *out) {
    if (!s || !out) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->inflight_bytes = s->inflight_bytes;
    return SOS_OK;
}

sos_status sos_server_replay(sos_server *s, int64_t n_req, const int32_t *stream_ids, const float *const *x_dev,
                             float *const *y_dev, const int64_t *n, const double *t_arrival, double *latency) {
    if (!s || n_req < 0 || (n_req > 0 && (!stream_ids || !x_dev || !y_dev || !n || !t_arrival || !latency)))
        return SOS_EINVAL;
    {
        // every request is checked before the first is queued: a chunk larger than the budget could
        // never be admitted, and the replay would not end
        std::lock_guard<std::mutex> lk(s->mu);
        for (int64_t j = 0; j < n_req; ++j) {
            const int sid = stream_ids[j];
            if (sid < 0 || sid >= static_cast<int>(s->streams.size()) || n[j] <= 0 || !x_dev[j] || !y_dev[j])
                return SOS_EINVAL;
            Req r;
            r.x = x_dev[j];
            r.y = y_dev[j];
            r.n = n[j];
            if (req_bytes(r) > s->cfg.budget_bytes) return SOS_EBUDGET;
        }
    }
    std::vector<uint64_t> ids(n_req, 0);
    const double t0 = now_s();
    int64_t i = 0;
    while (i < n_req) {
        const double t = now_s() - t0;
        if (t_arrival[i] > t) {
            const double wait = t_arrival[i] - t;
            if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
            continue;
        }
        // every request whose arrival time has passed, as one critical section
        std::lock_guard<std::mutex> lk(s->mu);
        for (; i < n_req && t_arrival[i] <= t; ++i) {
            const int sid = stream_ids[i];
            Req r;
            r.id = s->next_id++;
            r.sid = sid;
            r.x = x_dev[i];
            r.y = y_dev[i];
            r.n = n[i];
            r.t_submit = t0 + t_arrival[i];  // latency counts from the scheduled arrival
            ids[i] = r.id;
            Stream &st = s->streams[sid];
            if (!st.busy && st.q.empty()) s->ready.push_back(sid);
            st.q.push_back(r);
            s->queued += 1;
            s->stats.submitted += 1;
        }
        s->cv.notify_one();
    }
    // collect the completions of this replay
    int64_t got = 0;
    const uint64_t first = n_req ? ids[0] : 0;
    std::unique_lock<std::mutex> lk(s->mu_rec);
    while (got < n_req) {
        s->cv_rec.wait_for(lk, std::chrono::milliseconds(50), [&] { return !s->done.empty(); });
        for (const sos_completion &c : s->done) {
            const int64_t k = static_cast<int64_t>(c.request_id - first);
            if (k >= 0 && k < n_req && ids[k] == c.request_id) {
                latency[k] = c.t_done - c.t_submit;
                ++got;
            }
        }
        s->done.clear();
        if (s->sticky != SOS_OK) return static_cast<sos_status>(s->sticky.load());
    }
    return SOS_OK;
}

}  // extern "C"
