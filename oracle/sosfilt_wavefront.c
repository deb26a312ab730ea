/*
 * ORACLE -- test infrastructure only (host baseline).
 *
 * The oracle's recurrence run as the multi-core wavefront of Sec. III-A: the signal is cut into
 * groups of B samples, group g is carried through all K sections by thread g mod T, and before
 * section s it waits until group g-1 has left section s, whose state (z1, z2) it then continues.
 * Groups thus enter every section in order and each section sees its samples in order, with the
 * same transposed-direct-form-II update as oracle_sosfilt_f32 in float64, so the output and the
 * final state are bit-identical to the sequential oracle's (pinned in tests).  Threads on
 * different groups work on different sections at the same time, as in Sec. III-A.  Used
 * only as a multi-core host baseline beside the one-core oracle.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int K, T;
    const double *sos;
    double *z;                /* [K][2] state of each section, handed from group to group */
    const float *x;
    double *y;                /* NULL: outputs not kept (timing runs) */
    int64_t n, B, ng;
    _Atomic int64_t *done;    /* done[s]: groups that have left section s */
    _Atomic int failed;
    _Atomic int start;        /* set once the thread count T is final */
} wave_ctx;

typedef struct {
    wave_ctx *c;
    int tid;
} wave_arg;

static void *wave_worker(void *argp) {
    wave_arg *a = (wave_arg *)argp;
    wave_ctx *c = a->c;
    while (!atomic_load_explicit(&c->start, memory_order_acquire)) sched_yield();
    double *buf = (double *)malloc(sizeof(double) * (size_t)c->B);
    if (!buf) {
        atomic_store(&c->failed, 1);
        /* still pass every group this thread owns through the sections, so no one waits forever */
    }
    for (int64_t g = a->tid; g < c->ng; g += c->T) {
        const int64_t off = g * c->B;
        const int64_t len = (c->n - off) < c->B ? (c->n - off) : c->B;
        if (buf)
            for (int64_t i = 0; i < len; ++i) buf[i] = (double)c->x[off + i];
        for (int s = 0; s < c->K; ++s) {
            while (atomic_load_explicit(&c->done[s], memory_order_acquire) < g) sched_yield();
            if (buf) {
                const double *q = c->sos + 5 * s;
                double z1 = c->z[2 * s], z2 = c->z[2 * s + 1];
                for (int64_t i = 0; i < len; ++i) {
                    const double v = buf[i];
                    const double out = q[0] * v + z1;
                    z1 = q[1] * v - q[3] * out + z2;
                    z2 = q[2] * v - q[4] * out;
                    buf[i] = out;
                }
                c->z[2 * s] = z1;
                c->z[2 * s + 1] = z2;
            }
            atomic_store_explicit(&c->done[s], g + 1, memory_order_release);
        }
        if (buf && c->y) memcpy(c->y + off, buf, sizeof(double) * (size_t)len);
    }
    free(buf);
    return NULL;
}

/* y[n] (double, may be NULL) and zf[K][2] (may be NULL) for float32 input x, initial state zi
 * (NULL = zeros); groups of `block` samples on `threads` host threads. */
int oracle_sosfilt_wavefront_f32(int K, const double *sos, const float *x, int64_t n, const double *zi,
                                 double *y, double *zf, int64_t block, int threads) {
    if (K < 1 || n < 0 || block < 1) return -1;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    wave_ctx c;
    memset(&c, 0, sizeof c);
    c.K = K;
    c.T = threads;
    c.sos = sos;
    c.x = x;
    c.y = y;
    c.n = n;
    c.B = block;
    c.ng = (n + block - 1) / block;
    c.z = (double *)calloc((size_t)(2 * K), sizeof(double));
    c.done = (_Atomic int64_t *)calloc((size_t)K, sizeof(_Atomic int64_t));
    if (!c.z || !c.done) {
        free(c.z);
        free((void *)c.done);
        return -2;
    }
    if (zi) memcpy(c.z, zi, sizeof(double) * 2 * (size_t)K);
    for (int s = 0; s < K; ++s) atomic_init(&c.done[s], 0);
    atomic_init(&c.failed, 0);
    atomic_init(&c.start, 0);
    pthread_t tid[256];
    wave_arg args[256];
    int made = 0;
    for (int t = 1; t < threads; ++t) {
        args[t].c = &c;
        args[t].tid = t;
        if (pthread_create(&tid[made], NULL, wave_worker, &args[t]) != 0) break;
        ++made;
    }
    /* the groups are dealt over the threads that exist: T is final before any of them starts */
    c.T = made + 1;
    atomic_store_explicit(&c.start, 1, memory_order_release);
    args[0].c = &c;
    args[0].tid = 0;
    wave_worker(&args[0]);
    for (int t = 0; t < made; ++t) pthread_join(tid[t], NULL);
    const int failed = atomic_load(&c.failed);
    if (!failed && zf) memcpy(zf, c.z, sizeof(double) * 2 * (size_t)K);
    free(c.z);
    free((void *)c.done);
    return failed ? -2 : 0;
}
