/*
 * Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
 * benchmark.  This file holds no filtering arithmetic: it only draws numbers.
 *
 * Generator: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11),
 * written here from its published definition:
 *   round:  (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
 *                             hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
 *   key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85
 *   M0 = 0xD2511F53, M1 = 0xCD9E8D57, ten rounds.
 *
 * Stream layout: key = (seed low 32 bits, seed high 32 bits); the counter of
 * block i of stream s is (i low, i high, s low, s high).  Each block yields
 * four 32-bit words = two 64-bit words = two uniforms in (0,1) with 53-bit
 * resolution: u = ((w >> 11) + 0.5) * 2^-53.
 *
 * Normals: Box-Muller in double precision on the two uniforms of block i
 * (r = sqrt(-2 ln u0), z0 = r cos(2 pi u1), z1 = r sin(2 pi u1)), giving
 * samples 2i and 2i+1, then rounded to float32.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void wl_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

static void block_uniforms(uint64_t seed, uint64_t stream, uint64_t i, double u[2]) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    wl_philox4x32_10(ctr, key, o);
    uint64_t w0 = ((uint64_t)o[1] << 32) | o[0];
    uint64_t w1 = ((uint64_t)o[3] << 32) | o[2];
    u[0] = ((double)(w0 >> 11) + 0.5) * 0x1p-53;
    u[1] = ((double)(w1 >> 11) + 0.5) * 0x1p-53;
}

typedef struct {
    uint64_t seed, stream, n, begin, end; /* block range [begin, end) */
    int kind;                             /* 0 normal f32, 1 uniform f64 */
    float *out_f32;
    double *out_f64;
    double sin_amp, sin_omega; /* optional sinusoid added to the normals */
} wl_job;

static void *wl_worker(void *arg) {
    wl_job *j = (wl_job *)arg;
    const double two_pi = 6.283185307179586476925286766559;
    for (uint64_t i = j->begin; i < j->end; ++i) {
        double u[2];
        block_uniforms(j->seed, j->stream, i, u);
        uint64_t s0 = 2 * i, s1 = 2 * i + 1;
        if (j->kind == 1) {
            if (s0 < j->n) j->out_f64[s0] = u[0];
            if (s1 < j->n) j->out_f64[s1] = u[1];
        } else {
            double r = sqrt(-2.0 * log(u[0]));
            double z0 = r * cos(two_pi * u[1]);
            double z1 = r * sin(two_pi * u[1]);
            if (j->sin_amp != 0.0) {
                z0 += j->sin_amp * sin(j->sin_omega * (double)s0);
                z1 += j->sin_amp * sin(j->sin_omega * (double)s1);
            }
            if (s0 < j->n) j->out_f32[s0] = (float)z0;
            if (s1 < j->n) j->out_f32[s1] = (float)z1;
        }
    }
    return NULL;
}

static int wl_run(uint64_t seed, uint64_t stream, uint64_t n, int kind, float *of, double *od,
                  double sin_amp, double sin_omega, int threads) {
    uint64_t blocks = (n + 1) / 2;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (blocks < 65536) threads = 1;
    wl_job jobs[256];
    pthread_t tid[256];
    uint64_t per = (blocks + (uint64_t)threads - 1) / (uint64_t)threads;
    int started = 0;
    for (int t = 0; t < threads; ++t) {
        uint64_t b = (uint64_t)t * per, e = b + per;
        if (b > blocks) b = blocks;
        if (e > blocks) e = blocks;
        wl_job jb = {seed, stream, n, b, e, kind, of, od, sin_amp, sin_omega};
        jobs[t] = jb;
    }
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, wl_worker, &jobs[t]) != 0) {
            wl_worker(&jobs[t]); /* run inline if no thread could be made */
            tid[t] = 0;
        } else {
            ++started;
        }
    }
    wl_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t)
        if (tid[t]) pthread_join(tid[t], NULL);
    (void)started;
    return 0;
}

/* n float32 samples of N(0,1) (+ sin_amp * sin(sin_omega * k) at sample k). */
int wl_normal_f32(uint64_t seed, uint64_t stream, uint64_t n, float *out, double sin_amp,
                  double sin_omega, int threads) {
    return wl_run(seed, stream, n, 0, out, NULL, sin_amp, sin_omega, threads);
}

/* n uniforms in (0,1), double precision. */
int wl_uniform_f64(uint64_t seed, uint64_t stream, uint64_t n, double *out, int threads) {
    return wl_run(seed, stream, n, 1, NULL, out, 0.0, 0.0, threads);
}
