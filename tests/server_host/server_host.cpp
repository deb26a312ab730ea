// Host stand-ins for what the serving loop calls below it -- CUDA streams, memory and host
// functions, and the library's filter objects and batched run -- so that sosfilt_server.cpp's
// admission, ordering and completion logic runs on the CPU under test.  Test infrastructure only.
//
// A stream is a worker thread that runs its queued work in order.  A filter filters in float64
// through the transposed-direct-form-II cascade (Eq. 1) and keeps float32 states, as the library
// does between calls.  The batched run records how many batches and bytes were in flight at once.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <vector>

#include "cuda_runtime.h"
#include "sosfilt.h"

struct host_stream {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::function<void()>> q;
    bool busy = false, stop = false;
    std::thread worker;
    void loop() {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return stop || !q.empty(); });
            if (q.empty()) return;
            auto job = std::move(q.front());
            q.pop_front();
            busy = true;
            lk.unlock();
            job();
            lk.lock();
            busy = false;
            cv.notify_all();
        }
    }
    void push(std::function<void()> job) {
        {
            std::lock_guard<std::mutex> lk(mu);
            q.push_back(std::move(job));
        }
        cv.notify_all();
    }
};

struct sos_filter {
    int K = 0;
    std::vector<double> sos;
};

namespace {
std::mutex g_mu;
int g_batches_now = 0, g_batches_max = 0;
long long g_bytes_now = 0, g_bytes_max = 0, g_batches_total = 0;
int g_delay_us = 200;
int g_fail_next = 0;  // batched runs still to fail with SOS_ECUDA
}  // namespace

cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int *d) {
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaMalloc(void **p, size_t bytes) {
    *p = std::malloc(bytes ? bytes : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p) {
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind) {
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) {
    host_stream *h = new (std::nothrow) host_stream();
    if (!h) return cudaErrorMemoryAllocation;
    h->worker = std::thread([h] { h->loop(); });
    *s = h;
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t s) {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [&] { return s->q.empty() && !s->busy; });
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
    delete s;
    return cudaSuccess;
}
cudaError_t cudaLaunchHostFunc(cudaStream_t s, cudaHostFn_t fn, void *arg) {
    s->push([fn, arg] { fn(arg); });
    return cudaSuccess;
}

extern "C" {

sos_status sos_filter_create(int K, const double *sos, const float *, const sos_tuning *, sos_filter **out) {
    if (!out || !sos || K < 1) return SOS_EINVAL;
    sos_filter *f = new sos_filter();
    f->K = K;
    f->sos.assign(sos, sos + 5 * K);
    *out = f;
    return SOS_OK;
}
sos_status sos_filter_destroy(sos_filter *f) {
    delete f;
    return SOS_OK;
}

// Each signal through its cascade from state zi (float32 [K][2], NULL = zeros) to zf, on stream s.
sos_status sos_filter_run_batch_ex(int m, sos_filter *const *fs, const float *const *x, float *const *y,
                                   const int64_t *n, const float *const *zi, float *const *zf, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_fail_next > 0) {
            g_fail_next -= 1;
            return SOS_ECUDA;  // nothing enqueued, as when a launch is refused
        }
    }
    struct Sig {
        sos_filter *f;
        const float *x, *zi;
        float *y, *zf;
        int64_t n;
    };
    std::vector<Sig> sigs;
    long long bytes = 0;
    for (int i = 0; i < m; ++i) {
        sigs.push_back(Sig{fs[i], x[i], zi ? zi[i] : nullptr, y[i], zf ? zf[i] : nullptr, n[i]});
        bytes += (x[i] == y[i] ? 4 : 8) * n[i];
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_batches_now += 1;
        g_bytes_now += bytes;
        g_batches_total += 1;
        g_batches_max = std::max(g_batches_max, g_batches_now);
        g_bytes_max = std::max(g_bytes_max, g_bytes_now);
    }
    const int delay = g_delay_us;
    s->push([sigs, bytes, delay] {
        if (delay > 0) std::this_thread::sleep_for(std::chrono::microseconds(delay));
        for (const Sig &g : sigs) {
            const int K = g.f->K;
            std::vector<double> z(2 * K, 0.0);
            if (g.zi)
                for (int j = 0; j < 2 * K; ++j) z[j] = g.zi[j];
            for (int64_t t = 0; t < g.n; ++t) {
                double v = g.x[t];
                for (int k = 0; k < K; ++k) {
                    const double *c = &g.f->sos[5 * k];
                    const double out = c[0] * v + z[2 * k];
                    z[2 * k] = c[1] * v - c[3] * out + z[2 * k + 1];
                    z[2 * k + 1] = c[2] * v - c[4] * out;
                    v = out;
                }
                g.y[t] = static_cast<float>(v);
            }
            if (g.zf)
                for (int j = 0; j < 2 * K; ++j) g.zf[j] = static_cast<float>(z[j]);
        }
        std::lock_guard<std::mutex> lk(g_mu);
        g_batches_now -= 1;
        g_bytes_now -= bytes;
    });
    return SOS_OK;
}

// Test hooks: the largest number of batches and bytes in flight at once since the last reset, the
// batches run, the simulated run time of a batch, and batched runs made to fail.
void host_stats(long long *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    out[0] = g_batches_max;
    out[1] = g_bytes_max;
    out[2] = g_batches_total;
}
void host_fail_next(int n) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_fail_next = n;
}
void host_reset(int delay_us) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_fail_next = 0;
    g_batches_max = g_batches_now;
    g_bytes_max = g_bytes_now;
    g_batches_total = 0;
    g_delay_us = delay_us;
}

}  // extern "C"
