/*
 * Host-thread emulation of the lookback protocols of the PH kernels (a test aid; it shares no code
 * with the CUDA library).  Tiles are drawn from an ascending ticket counter by T worker threads
 * (Sec. IV-A).  Tile t publishes its local carry in slot 0 of its descriptor, tagged words of
 * (epoch << 2 | 1, float bits); it then composes its incoming state from the resolved carry of its
 * anchor tile a = 32 floor((t - 1) / 32) (slot 1, tag epoch << 2 | 2) and the local carries of
 * tiles a + 1 .. t - 1, with bounded spins, and an anchor tile publishes its resolved carry
 * A_T Z + local.  Tile 0 starts from z0.  A tile whose number equals `silent` never publishes
 * (failure injection): its successors' waits run out, set the status word and return.
 *
 * The composition is evaluated by Horner's rule from the anchor in float32, the same operations in
 * the same order as emu_reference(), so a correct protocol gives bit-identical results whatever
 * the interleaving of the threads.
 *
 * emu_run is the skewed-pass PH kernel's protocol.  The hierarchical form (emu_run_hier) is the
 * tensor-core kernel's: every tile first sums the
 * local carries after its anchor, P = sum_k A^(k-1) L(t - k) (Horner from zero); a tile between
 * anchors then forms G(a) itself, from the resolved carry of the super-anchor s below it and the
 * local parts of the anchors s + 32 .. a by the same Horner steps the anchor takes (so the bits
 * agree), and takes Z = A^(t-1-a) G(a) + P; an anchor t publishes its local part
 * W = A P + L(t) in its slot 0 (tag epoch << 2 | 3), waits for the resolved carry of the
 * super-anchor s below it (multiples of 128) and the local parts of the anchors between, composes
 * G(t) = A^32 (... (A^32 G(s) + W(s + 32)) ...) + W(t) by Horner's rule, publishes it and takes
 * Z = A^31 G(t - 32) + P.  The powers A^k are passed in (float32).
 *
 * The batched form (emu_run_batch) is the batch kernel's: the tiles of several signals share one
 * ticket queue (a tile -> signal map, each signal's tiles consecutive from its first tile t0), and
 * each signal keeps its own chain -- its first tile starts from the signal's initial state, the
 * anchors are t0 + 32 floor((t - 1 - t0) / 32), and its tiles compose with the signal's own
 * transition.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int S;
    int64_t n_tiles;
    unsigned epoch;
    _Atomic uint64_t *desc;  /* [n_tiles][2][S] */
    const float *local;      /* [n_tiles][S] local carries */
    const float *AT;         /* [signals][S][S] row-major tile transition of each signal */
    const float *APow;       /* hierarchical protocol: [33][S][S] A^k, k = 0 .. 32; else NULL */
    const float *z0;         /* [signals][S] initial state of each signal */
    const int *tile_sig;     /* [n_tiles] signal of each tile */
    const int64_t *tile0;    /* [signals] first tile of each signal */
    float *Z;                /* [n_tiles][S] incoming states (output) */
    _Atomic int64_t ticket;
    _Atomic int status;      /* 1: a wait ran out */
    int64_t spin_limit;      /* polls before a wait gives up */
    int64_t silent;          /* tile that never publishes, or -1 */
} emu_ctx;

static uint64_t pack(unsigned tag, float v) {
    uint32_t b;
    memcpy(&b, &v, sizeof b);
    return ((uint64_t)tag << 32) | b;
}

static float payload(uint64_t w) {
    uint32_t b = (uint32_t)w;
    float v;
    memcpy(&v, &b, sizeof v);
    return v;
}

/* y = A x (S x S row-major), then y += b */
static void mv_add(int S, const float *A, const float *x, const float *b, float *y) {
    for (int i = 0; i < S; ++i) {
        float acc = 0.f;
        for (int j = 0; j < S; ++j) acc = acc + A[i * S + j] * x[j];
        y[i] = acc + b[i];
    }
}

/* Waits until every word of the S-word slot carries `tag` and copies the payloads; 0 on timeout. */
static int wait_slot(emu_ctx *c, int64_t tile, int slot, unsigned tag, float *out) {
    _Atomic uint64_t *w = c->desc + ((size_t)tile * 2 + (size_t)slot) * (size_t)c->S;
    for (int64_t spin = 0;; ++spin) {
        int ok = 1;
        for (int i = 0; i < c->S; ++i) {
            const uint64_t v = atomic_load_explicit(&w[i], memory_order_acquire);
            if ((unsigned)(v >> 32) != tag) {
                ok = 0;
                break;
            }
            out[i] = payload(v);
        }
        if (ok) return 1;
        if (spin >= c->spin_limit) return 0;
        sched_yield();
    }
}

static void publish(emu_ctx *c, int64_t tile, int slot, unsigned tag, const float *v) {
    _Atomic uint64_t *w = c->desc + ((size_t)tile * 2 + (size_t)slot) * (size_t)c->S;
    for (int i = 0; i < c->S; ++i) atomic_store_explicit(&w[i], pack(tag, v[i]), memory_order_release);
}

/* The hierarchical composition of tile t (single signal); 0 when a wait ran out. */
static int hier_tile(emu_ctx *c, int64_t t) {
    const int S = c->S;
    const unsigned tagL = (c->epoch << 2) | 1u, tagG = (c->epoch << 2) | 2u, tagW = (c->epoch << 2) | 3u;
    const float *A = c->AT, *AP = c->APow;
    const float *loc = c->local + (size_t)t * S;
    const int anchor = t % 32 == 0 && t + 1 < c->n_tiles;
    float P[64], v[64], tmp[64], h[64], g[64];
    if (!anchor && t > 0) publish(c, t, 0, tagL, loc);
    if (t == 0) {
        memcpy(c->Z, c->z0, sizeof(float) * (size_t)S);
        if (anchor) {
            mv_add(S, A, c->z0, loc, tmp);
            publish(c, 0, 1, tagG, tmp);
        }
        return 1;
    }
    const int64_t a = ((t - 1) / 32) * 32;
    memset(P, 0, sizeof(float) * (size_t)S);
    for (int64_t p = a + 1; p < t; ++p) {
        if (!wait_slot(c, p, 0, tagL, v)) return 0;
        mv_add(S, A, P, v, tmp);
        memcpy(P, tmp, sizeof(float) * (size_t)S);
    }
    if (!anchor) {
        /* G(a) formed here from the super-anchor's resolved carry and the anchors' local parts */
        const int64_t s0 = ((t - 1) / 128) * 128;
        if (!wait_slot(c, s0, 1, tagG, g)) return 0;
        for (int64_t b = s0 + 32; b <= a; b += 32) {
            if (!wait_slot(c, b, 0, tagW, v)) return 0;
            mv_add(S, AP + (size_t)32 * S * S, g, v, tmp);
            memcpy(g, tmp, sizeof(float) * (size_t)S);
        }
        mv_add(S, AP + (size_t)(t - 1 - a) * S * S, g, P, c->Z + (size_t)t * S);
        return 1;
    }
    float W[64];
    mv_add(S, A, P, loc, W);
    publish(c, t, 0, tagW, W);
    const int64_t s0 = ((t - 1) / 128) * 128;
    if (!wait_slot(c, s0, 1, tagG, h)) return 0;
    for (int64_t b = s0 + 32; b < t; b += 32) {
        if (!wait_slot(c, b, 0, tagW, v)) return 0;
        mv_add(S, AP + (size_t)32 * S * S, h, v, tmp);
        memcpy(h, tmp, sizeof(float) * (size_t)S);
    }
    mv_add(S, AP + (size_t)32 * S * S, h, W, tmp);
    publish(c, t, 1, tagG, tmp);
    mv_add(S, AP + (size_t)31 * S * S, h, P, c->Z + (size_t)t * S);
    return 1;
}

static void *emu_worker(void *arg) {
    emu_ctx *c = (emu_ctx *)arg;
    const int S = c->S;
    const unsigned tagL = (c->epoch << 2) | 1u, tagG = (c->epoch << 2) | 2u;
    float acc[64], v[64], tmp[64];
    for (;;) {
        const int64_t t = atomic_fetch_add(&c->ticket, 1);
        if (t >= c->n_tiles || atomic_load(&c->status)) break;
        if (t == c->silent) continue;  /* this tile's worker "dies" before publishing anything */
        if (c->APow) {
            if (!hier_tile(c, t)) {
                atomic_store(&c->status, 1);
                break;
            }
            continue;
        }
        const int sig = c->tile_sig[t];
        const int64_t t0 = c->tile0[sig];
        const float *A = c->AT + (size_t)sig * S * S;
        const float *loc = c->local + (size_t)t * S;
        if (t > t0) publish(c, t, 0, tagL, loc);
        if (t == t0) {
            memcpy(acc, c->z0 + (size_t)sig * S, sizeof(float) * (size_t)S);
        } else {
            const int64_t a = t0 + ((t - 1 - t0) / 32) * 32;
            if (!wait_slot(c, a, 1, tagG, acc)) {
                atomic_store(&c->status, 1);
                break;
            }
            for (int64_t p = a + 1; p < t; ++p) {
                if (!wait_slot(c, p, 0, tagL, v)) {
                    atomic_store(&c->status, 1);
                    return NULL;
                }
                mv_add(S, A, acc, v, tmp);
                memcpy(acc, tmp, sizeof(float) * (size_t)S);
            }
        }
        memcpy(c->Z + (size_t)t * S, acc, sizeof(float) * (size_t)S);
        if ((t - t0) % 32 == 0 && t + 1 < c->n_tiles) {
            mv_add(S, A, acc, loc, tmp);
            publish(c, t, 1, tagG, tmp);
        }
    }
    return NULL;
}

/* One launch of the batched protocol over `desc` (kept by the caller between launches: its old
 * tags must not be mistaken for this epoch's).  Returns 0, or 1 when some wait ran out. */
static int emu_launch(int S, int64_t n_tiles, unsigned epoch, uint64_t *desc, const float *local, const float *AT,
                      const float *APow, const float *z0, const int *tile_sig, const int64_t *tile0, float *Z,
                      int threads, int64_t spin_limit, int64_t silent) {
    if (S < 1 || S > 64 || n_tiles < 0 || threads < 1 || threads > 64) return -1;
    emu_ctx c;
    memset(&c, 0, sizeof c);
    c.S = S;
    c.n_tiles = n_tiles;
    c.epoch = epoch;
    c.desc = (_Atomic uint64_t *)desc;
    c.local = local;
    c.AT = AT;
    c.APow = APow;
    c.z0 = z0;
    c.tile_sig = tile_sig;
    c.tile0 = tile0;
    c.Z = Z;
    atomic_init(&c.ticket, 0);
    atomic_init(&c.status, 0);
    c.spin_limit = spin_limit;
    c.silent = silent;
    pthread_t tid[64];
    int made = 0;
    for (int i = 1; i < threads; ++i)
        if (pthread_create(&tid[made], NULL, emu_worker, &c) == 0) ++made;
    emu_worker(&c);
    for (int i = 0; i < made; ++i) pthread_join(tid[i], NULL);
    return atomic_load(&c.status);
}

int emu_run_batch(int S, int64_t n_tiles, unsigned epoch, uint64_t *desc, const float *local, const float *AT,
                  const float *z0, const int *tile_sig, const int64_t *tile0, float *Z, int threads,
                  int64_t spin_limit, int64_t silent) {
    return emu_launch(S, n_tiles, epoch, desc, local, AT, NULL, z0, tile_sig, tile0, Z, threads, spin_limit, silent);
}

/* One signal, hierarchical protocol (APow: A^k, k = 0 .. 32). */
int emu_run_hier(int S, int64_t n_tiles, unsigned epoch, uint64_t *desc, const float *local, const float *AT,
                 const float *APow, const float *z0, float *Z, int threads, int64_t spin_limit, int64_t silent) {
    if (n_tiles < 0 || !APow) return -1;
    int *ts = (int *)calloc((size_t)(n_tiles > 0 ? n_tiles : 1), sizeof(int));
    if (!ts) return -1;
    const int64_t t0 = 0;
    const int rc = emu_launch(S, n_tiles, epoch, desc, local, AT, APow, z0, ts, &t0, Z, threads, spin_limit, silent);
    free(ts);
    return rc;
}

/* The hierarchical composition, tile after tile on one thread (the same operations in the same
 * order as hier_tile). */
void emu_reference_hier(int S, int64_t n_tiles, const float *local, const float *A, const float *AP, const float *z0,
                        float *Z) {
    float *Wv = (float *)calloc((size_t)S * (size_t)(n_tiles > 0 ? n_tiles : 1), sizeof(float));
    float *Gv = (float *)calloc((size_t)S * (size_t)(n_tiles > 0 ? n_tiles : 1), sizeof(float));
    float P[64], tmp[64], h[64];
    for (int64_t t = 0; t < n_tiles; ++t) {
        const float *loc = local + (size_t)t * S;
        const int anchor = t % 32 == 0 && t + 1 < n_tiles;
        if (t == 0) {
            memcpy(Z, z0, sizeof(float) * (size_t)S);
            if (anchor) mv_add(S, A, z0, loc, Gv);
            continue;
        }
        const int64_t a = ((t - 1) / 32) * 32;
        memset(P, 0, sizeof(float) * (size_t)S);
        for (int64_t p = a + 1; p < t; ++p) {
            mv_add(S, A, P, local + (size_t)p * S, tmp);
            memcpy(P, tmp, sizeof(float) * (size_t)S);
        }
        if (!anchor) {
            mv_add(S, AP + (size_t)(t - 1 - a) * S * S, Gv + (size_t)a * S, P, Z + (size_t)t * S);
            continue;
        }
        float *W = Wv + (size_t)t * S;
        mv_add(S, A, P, loc, W);
        const int64_t s0 = ((t - 1) / 128) * 128;
        memcpy(h, Gv + (size_t)s0 * S, sizeof(float) * (size_t)S);
        for (int64_t b = s0 + 32; b < t; b += 32) {
            mv_add(S, AP + (size_t)32 * S * S, h, Wv + (size_t)b * S, tmp);
            memcpy(h, tmp, sizeof(float) * (size_t)S);
        }
        mv_add(S, AP + (size_t)32 * S * S, h, W, Gv + (size_t)t * S);
        mv_add(S, AP + (size_t)31 * S * S, h, P, Z + (size_t)t * S);
    }
    free(Wv);
    free(Gv);
}

/* One signal: every tile maps to signal 0, whose first tile is 0. */
int emu_run(int S, int64_t n_tiles, unsigned epoch, uint64_t *desc, const float *local, const float *AT,
            const float *z0, float *Z, int threads, int64_t spin_limit, int64_t silent) {
    if (n_tiles < 0) return -1;
    int *ts = (int *)calloc((size_t)(n_tiles > 0 ? n_tiles : 1), sizeof(int));
    if (!ts) return -1;
    const int64_t t0 = 0;
    const int rc = emu_run_batch(S, n_tiles, epoch, desc, local, AT, z0, ts, &t0, Z, threads, spin_limit, silent);
    free(ts);
    return rc;
}

/* The same composition evaluated signal by signal, tile after tile, on one thread. */
void emu_reference_batch(int S, int n_signals, const int64_t *tile0, const int64_t *n_sig_tiles, const float *local,
                         const float *AT, const float *z0, float *Z) {
    float acc[64], tmp[64];
    for (int sig = 0; sig < n_signals; ++sig) {
        const int64_t t0 = tile0[sig], nt = n_sig_tiles[sig];
        const float *A = AT + (size_t)sig * S * S;
        float *res = (float *)malloc(sizeof(float) * (size_t)S * (size_t)(nt > 0 ? nt : 1));
        for (int64_t r = 0; r < nt; ++r) {  /* r: tile number within the signal */
            if (r == 0) {
                memcpy(acc, z0 + (size_t)sig * S, sizeof(float) * (size_t)S);
            } else {
                const int64_t a = ((r - 1) / 32) * 32;
                memcpy(acc, res + (size_t)a * S, sizeof(float) * (size_t)S);
                for (int64_t p = a + 1; p < r; ++p) {
                    mv_add(S, A, acc, local + (size_t)(t0 + p) * S, tmp);
                    memcpy(acc, tmp, sizeof(float) * (size_t)S);
                }
            }
            memcpy(Z + (size_t)(t0 + r) * S, acc, sizeof(float) * (size_t)S);
            if (r % 32 == 0) mv_add(S, A, acc, local + (size_t)(t0 + r) * S, res + (size_t)r * S);
        }
        free(res);
    }
}

void emu_reference(int S, int64_t n_tiles, const float *local, const float *AT, const float *z0, float *Z) {
    const int64_t t0 = 0;
    emu_reference_batch(S, 1, &t0, &n_tiles, local, AT, z0, Z);
}
