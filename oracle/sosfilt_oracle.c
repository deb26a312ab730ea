/*
 * ORACLE -- test infrastructure only.
 *
 * Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this code.  The GPU library shares nothing with it.
 *
 * What it computes: the cascade of K second-order sections of Eq. 1 (Sec. II-A),
 * run sample by sample in float64, in the transposed direct form II:
 *
 *     y     = b0*x + z1
 *     z1   <- b1*x - a1*y + z2
 *     z2   <- b2*x - a2*y
 *
 * per section k = 0..K-1 in order, where the output of section k is the input
 * of section k+1.  This is the plain definition of the filter: the
 * multi-block system of Eq. 2 has exactly this solution, so the GPU result
 * may differ from it only by float32 rounding.  The initial state zi[k] =
 * (z1, z2) and the final state zf[k] use the same convention.  Input samples
 * are float32 widened to double (or double, for tests); coefficients are
 * double.  sos is [K][5] = b0, b1, b2, a1, a2 with a0 = 1.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static void cascade_f64(int K, const double *sos, double *z, const void *x, int x_is_f32, int64_t n,
                        double *y) {
    for (int64_t i = 0; i < n; ++i) {
        double v = x_is_f32 ? (double)((const float *)x)[i] : ((const double *)x)[i];
        for (int k = 0; k < K; ++k) {
            const double *c = sos + 5 * k;
            double *s = z + 2 * k;
            double out = c[0] * v + s[0];
            s[0] = c[1] * v - c[3] * out + s[1];
            s[1] = c[2] * v - c[4] * out;
            v = out;
        }
        if (y) y[i] = v;
    }
}

static int prepare_state(int K, const double *zi, double **z) {
    *z = (double *)calloc((size_t)(2 * K), sizeof(double));
    if (!*z) return -1;
    if (zi) memcpy(*z, zi, sizeof(double) * 2 * (size_t)K);
    return 0;
}

/* y[n] (double) and zf[K][2] (may be NULL) for float32 input x. */
int oracle_sosfilt_f32(int K, const double *sos, const float *x, int64_t n, const double *zi,
                       double *y, double *zf) {
    if (K < 1 || n < 0) return -1;
    double *z;
    if (prepare_state(K, zi, &z)) return -2;
    cascade_f64(K, sos, z, x, 1, n, y);
    if (zf) memcpy(zf, z, sizeof(double) * 2 * (size_t)K);
    free(z);
    return 0;
}

/* Same for double input. */
int oracle_sosfilt_f64(int K, const double *sos, const double *x, int64_t n, const double *zi,
                       double *y, double *zf) {
    if (K < 1 || n < 0) return -1;
    double *z;
    if (prepare_state(K, zi, &z)) return -2;
    cascade_f64(K, sos, z, x, 0, n, y);
    if (zf) memcpy(zf, z, sizeof(double) * 2 * (size_t)K);
    free(z);
    return 0;
}

/*
 * Many independent signals, one per task, spread over `threads` host threads
 * (signals are independent; each one is still the sequential recurrence).
 * Signal s uses K[s] sections at sos + 5*sos_off[s], input x + x_off[s] of
 * length n[s], writes y + x_off[s] and zf + 2*sos_off[s]; zero initial state.
 */
typedef struct {
    int n_signals;
    const int *K;
    const int64_t *sos_off, *x_off, *n;
    const double *sos;
    const float *x;
    double *y, *zf;
    int64_t next;
    pthread_mutex_t mu;
} batch_ctx;

static void *batch_worker(void *arg) {
    batch_ctx *c = (batch_ctx *)arg;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        int64_t s = c->next++;
        pthread_mutex_unlock(&c->mu);
        if (s >= c->n_signals) break;
        double *zf = c->zf ? c->zf + 2 * c->sos_off[s] : NULL;
        oracle_sosfilt_f32(c->K[s], c->sos + 5 * c->sos_off[s], c->x + c->x_off[s], c->n[s], NULL,
                           c->y ? c->y + c->x_off[s] : NULL, zf);
    }
    return NULL;
}

int oracle_sosfilt_batch_f32(int n_signals, const int *K, const int64_t *sos_off, const double *sos,
                             const int64_t *x_off, const int64_t *n, const float *x, double *y,
                             double *zf, int threads) {
    if (n_signals < 0) return -1;
    if (threads < 1) threads = 1;
    if (threads > 512) threads = 512;
    batch_ctx c;
    memset(&c, 0, sizeof c);
    c.n_signals = n_signals;
    c.K = K;
    c.sos_off = sos_off;
    c.x_off = x_off;
    c.n = n;
    c.sos = sos;
    c.x = x;
    c.y = y;
    c.zf = zf;
    c.next = 0;
    pthread_mutex_init(&c.mu, NULL);
    pthread_t tid[512];
    int made = 0;
    for (int t = 1; t < threads; ++t)
        if (pthread_create(&tid[made], NULL, batch_worker, &c) == 0) ++made;
    batch_worker(&c);
    for (int t = 0; t < made; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&c.mu);
    return 0;
}
