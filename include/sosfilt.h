/*
 * sosfilt.h -- C ABI of libsosfilt.so: cascaded second-order IIR filtering of
 * long float32 signals on one GB300 GPU (sm_103a).
 *
 * Method (Zhai & Paris, "Parallel Cascaded Recursive Filtering on Multi-Core
 * CPUs and GPUs"): every group of C = N*L samples is stride-N permuted into the
 * block-banded system of Eq. 2-3 (Sec. II-B).  Its zero-state response is
 * solved in registers, by default by PH factorization (Sec. II-C: per-lane
 * particular solutions and a lane scan), or, selected by sos_tuning.solver, by
 * divide-and-conquer cyclic reduction (Sec. II-D, II-E, Eqs. 14-23), which
 * exposes both terminal samples of a lane before back substitution.  Terminal
 * states are carried across groups by decoupled lookback (Sec. IV-B, Eq. 25) and
 * the homogeneous correction (Eq. 24) is applied once a group's incoming state
 * is known.  All K sections of a group stay in registers inside one kernel
 * (Sec. IV-A).
 *
 * Conventions used by every entry point
 *   - Coefficients: `sos` is a host array [n_sections][5] of double holding
 *     b0, b1, b2, a1, a2 per section, a0 = 1 (Eq. 1 with the section gain b0
 *     kept per section).  Section k's output is section k+1's input.
 *   - State: [n_sections][2] float32 in transposed direct form II, the
 *     convention of scipy.signal.sosfilt: after a sample x with output y,
 *         z1 = b1*x - a1*y + z2_old,   z2 = b2*x - a2*y.
 *     (Sec. II-B carries the last two inputs and outputs instead; both fix
 *     the same future outputs: (z1, z2) is exactly the forcing B_ x_-1 - A_ y_-1
 *     on the first two rows of Eq. 2.)
 *   - Samples are float32; arithmetic is float32 (tables are derived in
 *     float64 on the host and rounded once).
 *   - Device pointers are plain CUDA device addresses (e.g. torch tensors'
 *     data_ptr()).  `stream` is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  Every call that takes a stream is asynchronous
 *     on it; argument errors are returned synchronously; device-side errors
 *     (a lookback wait that ran out of time) set a sticky status read by
 *     sos_filter_sync_status().
 *   - Thread safety: a filter object may be used by one host thread and one
 *     stream at a time; different filter objects are independent.
 */
#ifndef SOSFILT_H
#define SOSFILT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SOS_OK = 0,
    SOS_EINVAL = -1,    /* bad argument: NULL where not allowed, n < 0, K out of range, overlap */
    SOS_ENOMEM = -2,    /* device or host allocation failed */
    SOS_ECUDA = -3,     /* a CUDA runtime call failed (launch, copy, device query) */
    SOS_ETIMEOUT = -4,  /* a lookback wait exceeded its cycle budget on the device */
    SOS_EUNSTABLE = -5, /* a section violates |a2| < 1, |a1| < 1 + a2, or a coefficient is not finite */
    SOS_EBUDGET = -6    /* the request exceeds the memory budget of the caller's setting */
} sos_status;

/* Opaque filter object, owned by the library. */
typedef struct sos_filter sos_filter;

/* Carry schemes (see sos_tuning.carry). */
enum {
    SOS_CARRY_DEFAULT = 0, /* SOS_CARRY_CASCADE */
    SOS_CARRY_CASCADE = 1, /* one carry per tile for the whole cascade state (2K words): a
                              zero-state pass through all sections, one decoupled lookback
                              (Sec. IV-B, Eq. 25 on the cascade state), then the homogeneous
                              correction of Eq. 24 applied once to the output */
    SOS_CARRY_SECTION = 2  /* one decoupled lookback per section, as in Sec. IV-B */
};

/* Solvers of a group's zero-state response (see sos_tuning.solver). */
enum {
    SOS_SOLVER_DEFAULT = 0, /* the library's choice: SOS_SOLVER_PH, or SOS_SOLVER_CR when the
                               tuning sets a carry scheme, a lookback width or N = 128 */
    SOS_SOLVER_CR = 1,      /* divide-and-conquer cyclic reduction per section (Sec. II-D, II-E,
                               Eqs. 14-23); both carry schemes */
    SOS_SOLVER_PH = 2,      /* PH factorization (Sec. II-C): per-lane particular solutions from zero
                               state (the sections skewed one sample apart so that their updates
                               are independent), a lane scan of the whole cascade state and one
                               homogeneous correction for lane and group states; cascade carry
                               only, N = 32 or 64 (default 64) */
    SOS_SOLVER_DTCR = 3,    /* double-thread-group cyclic reduction (Sec. IV-E): cyclic reduction
                               with the even- and odd-parity chains of every group on two warps,
                               exchanging through shared memory at each section (two barriers per
                               section); cascade carry only, N = 64 (tiles of four groups) */
    SOS_SOLVER_TC = 4       /* PH factorization (Sec. II-C) on the tensor cores: a lane's particular
                               solution is its 64 samples times the lower-triangular Toeplitz matrix
                               of the cascade's first 64 impulse-response taps (the inverse of the
                               lane's band matrix), its terminal state the product with the 64 state
                               responses, and the homogeneous correction (Eq. 24) the product of the
                               lanes' true states with the output basis; TF32 products with every
                               float32 operand split into head and remainder (float32 accuracy).
                               Cascade carry only, N = 64, tiles of 8 groups.  Needs x and y
                               16-byte aligned and n >= 64; other runs use SOS_SOLVER_PH */
};

/*
 * Launch configuration.  Any field left 0 selects the library's default for
 * that field (the built-in per-order table).
 *   N                  samples per thread (block count of Eq. 2): 32 or 64 for
 *                      the cascade carry; 32, 64 or 128 for per-section carries
 *   L                  threads per group (block length of Eq. 2): 32
 *   groups_per_cta     groups (compute warps, one per group) per thread block and tile:
 *                      0 = the library's choice (the autotuner's, else 7 for PH and the
 *                      carry scheme's fixed count for cyclic reduction); the PH solver
 *                      also takes 7, or 10 at N = 64 (11 warps per block: three warps on
 *                      most SM schedulers instead of two, a two-sample-wide correction
 *                      to stay within 168 registers); any other solver: 0
 *   threads_per_group  L (one thread group per signal block group, Sec. IV-D)
 *   fp64_carry         reserved: must be 0 (carries are float32)
 *   spin_budget_cycles upper bound, in SM clock cycles, on one lookback wait;
 *                      on expiry the kernel records SOS_ETIMEOUT and returns
 *   lookback_width     per-section carries only: predecessors read per lookback
 *                      round, in units of 32: 1, 2, 4, 8 or 16 (values other than
 *                      the default for N exist for 8-section passes with b0 != 0)
 *   carry              SOS_CARRY_DEFAULT, SOS_CARRY_CASCADE or SOS_CARRY_SECTION
 *   solver             SOS_SOLVER_DEFAULT, SOS_SOLVER_CR, SOS_SOLVER_PH, SOS_SOLVER_DTCR or
 *                      SOS_SOLVER_TC (see SOS_SOLVER_*); SOS_SOLVER_PH takes N = 0, 32 or 64,
 *                      SOS_SOLVER_DTCR and SOS_SOLVER_TC N = 0 or 64, all three carry
 *                      SOS_CARRY_DEFAULT or SOS_CARRY_CASCADE and lookback_width 0
 *   deterministic      0 or 1.  The PH solvers (and batched runs) always compose a tile's
 *                      incoming state the same way -- the resolved carry of a fixed anchor tile
 *                      (the last multiple of 32 before it) and the local carries after it -- so
 *                      their outputs are bit-identical from run to run.  Cyclic reduction composes
 *                      from whichever predecessor's resolved carry its lookback meets first (Sec.
 *                      IV-B) and may differ in the last ulps; 1 requests reproducible results and
 *                      is rejected with SOS_EINVAL together with solver SOS_SOLVER_CR or
 *                      SOS_SOLVER_DTCR, a carry other than SOS_CARRY_DEFAULT, a lookback width or
 *                      N = 128.
 */
typedef struct {
    int N, L, groups_per_cta, threads_per_group, fp64_carry;
    long long spin_budget_cycles;
    int lookback_width;
    int carry;
    int solver;
    int deterministic;
} sos_tuning;

/*
 * Create a filter from K = n_sections sections (Eq. 1).
 *   sos  host [K][5] double: b0, b1, b2, a1, a2 (copied; caller keeps ownership)
 *   zi   host [K][2] float32 initial resident state for sos_filter_stream_push
 *        (NULL = zeros)
 *   t    host tuning (NULL = defaults)
 *   out  receives the new filter; *out is NULL on failure
 * Errors: SOS_EINVAL (K < 1 or K > 64, NULL sos/out, bad tuning),
 * SOS_EUNSTABLE (a section outside the stability triangle or not finite),
 * SOS_ENOMEM, SOS_ECUDA.  Allocates device memory on the current device.
 */
sos_status sos_filter_create(int n_sections, const double *sos, const float *zi, const sos_tuning *t,
                             sos_filter **out);

/* Release a filter and its device memory.  NULL is a no-op.  Synchronizes the
 * device (every stream) before freeing, so that no enqueued run still reads it. */
sos_status sos_filter_destroy(sos_filter *f);

/*
 * Filter one signal: y = cascade(x), Sec. II and Sec. IV (one kernel launch
 * per pass of up to 8 sections).
 *   x_dev   device float32[n] input, contiguous
 *   y_dev   device float32[n] output, contiguous; y_dev == x_dev (in place) is
 *           allowed, any other overlap is SOS_EINVAL
 *   n       number of samples, >= 0; n = 0 only copies zi to zf
 *   zi_dev  device float32[K][2] initial state or NULL (zeros)
 *   zf_dev  device float32[K][2] receives the final state, or NULL; may equal zi_dev
 *   stream  cudaStream_t as void*
 * Ownership: the caller owns x, y, zi, zf; the library owns its workspace
 * (lookback descriptors, ticket counter, status word), grown on demand.
 * CUDA graphs: a run may be captured into a graph on `stream` (solvers PH, DTCR and
 * cyclic reduction with the cascade carry; per-section carries give SOS_EINVAL).
 * A captured run resets its own ticket counter and lookback descriptors inside the
 * graph, so every replay starts afresh; it allocates nothing, so the filter must
 * have run once outside the capture on a signal at least as long (else SOS_EINVAL).
 * Replays must not overlap each other or other runs of the same filter.
 */
sos_status sos_filter_run(sos_filter *f, const float *x_dev, float *y_dev, int64_t n, const float *zi_dev,
                          float *zf_dev, void *stream);

/*
 * Filter a signal held in HOST memory.  Synchronous: returns when y_host holds
 * the output.  Two ways, chosen by chunk_samples:
 *   staged (chunk_samples >= 0): the library copies the signal to the device,
 *     filters it and copies the result back in chunks, overlapping the
 *     host->device copy of chunk i+1, the filtering of chunk i (sos_filter_run
 *     with the state carried on the device from chunk to chunk, so the output
 *     equals one call over the whole signal) and the device->host copy of
 *     chunk i-1 on three library streams;
 *   direct (chunk_samples == SOS_HOST_DIRECT): the kernels read x_host and
 *     write y_host where they are, through their device mappings, in one run:
 *     no device buffers and no staging copies.  The buffers must be pinned
 *     (cudaHostAlloc, torch's pin_memory) or registered (cudaHostRegister);
 *     other host memory is SOS_EINVAL.
 *   x_host, y_host  host float32[n]; may be equal, any other overlap is SOS_EINVAL;
 *                   pinned memory lets the staged copies run at full speed
 *   zi_host         host float32[K][2] initial state or NULL (zeros)
 *   zf_host         host float32[K][2] receives the final state, or NULL
 *   chunk_samples   staged: samples per chunk, 0 = 2^24; the library keeps three
 *                   device buffers of this size per filter after the first call
 * Errors: SOS_EINVAL, SOS_ENOMEM, SOS_ECUDA; SOS_ETIMEOUT when a device wait of this call (or of
 * an earlier unreported run) ran out of time, reported and cleared as by sos_filter_sync_status.
 */
#define SOS_HOST_DIRECT (-1LL)
sos_status sos_filter_run_host(sos_filter *f, const float *x_host, float *y_host, int64_t n, const float *zi_host,
                               float *zf_host, int64_t chunk_samples);

/*
 * Filter many independent signals of uneven length and order in one persistent
 * kernel launch on `stream`: the signals with the same section count, the same
 * b0 handling and the same tile geometry form a class with its own global
 * queue of (signal, tile) work items, with the lookback chains of Sec. IV-B
 * kept per signal (a chain ends at its signal's first tile); each thread block
 * starts on a class in proportion to the classes' work and then takes every
 * other class that still has tiles.  Tile geometry per signal: 7 groups of
 * 32 x 64 samples (N = 64) or of 32 x 32 samples (N = 32), L = 32 threads per
 * group either way -- the filter's tuning N when it is 32 or 64, else the
 * choice of sos_autotune_batch for the signal's section count and length when
 * it has run on the device, else N = 64.  Zero initial state for every
 * signal.
 *   n_signals  >= 0
 *   filters    host array [n_signals] of filter objects (may repeat), all on one device
 *   x_dev      host array [n_signals] of device input pointers
 *   y_dev      host array [n_signals] of device output pointers (in place allowed)
 *   n          host array [n_signals] of lengths (>= 0)
 * Filters of more than 8 sections are filtered one by one (sos_filter_run).
 * The library keeps eight scratch sets per device (signal descriptors, lookback
 * descriptors); a call waits on the host until the device has finished the
 * batch that used its scratch set eight calls earlier, so batch calls must not
 * be made while `stream` is being captured into a CUDA graph.  Calls on one
 * device are serialized on the host.  Device-side errors: sos_batch_sync_status.
 */
sos_status sos_filter_run_batch(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                float *const *y_dev, const int64_t *n, void *stream);

/*
 * sos_filter_run_batch with an initial and a final state per signal (the form
 * the serving loop uses to keep every stream's cascade state on the device).
 *   zi_dev  host array [n_signals] of device float32[K][2] initial states, or
 *           NULL (all zero); an entry may be NULL (zero)
 *   zf_dev  host array [n_signals] of device float32[K][2] final states, or NULL;
 *           an entry may be NULL.  zf_dev[i] must not alias zi_dev[i].
 */
sos_status sos_filter_run_batch_ex(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                   float *const *y_dev, const int64_t *n, const float *const *zi_dev,
                                   float *const *zf_dev, void *stream);

/*
 * A prepared batch for repeated runs and CUDA graphs: the signal descriptors
 * and lookback workspace of a fixed set of signals (arguments as
 * sos_filter_run_batch_ex; every n > 0, at most 8 sections per filter) are
 * uploaded once.  sos_batch_plan_launch enqueues the batch on `stream` with no
 * host synchronization and no host-side work per signal (a reset of the
 * plan's descriptors and tickets, then the one persistent launch over every
 * class), so it may be captured into a CUDA graph and the graph replayed.  Launches of one plan
 * must not overlap on the device (they share its workspace).  The buffers and
 * filters named at creation must outlive the plan.
 */
typedef struct sos_batch_plan sos_batch_plan;
sos_status sos_batch_plan_create(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                 float *const *y_dev, const int64_t *n, const float *const *zi_dev,
                                 float *const *zf_dev, sos_batch_plan **out);
sos_status sos_batch_plan_launch(sos_batch_plan *plan, void *stream);
/* Synchronize the device and return the plan's sticky device status. */
sos_status sos_batch_plan_status(sos_batch_plan *plan);
/* Synchronizes the device, then releases the plan. */
sos_status sos_batch_plan_destroy(sos_batch_plan *plan);

/* Synchronize the device and return the sticky status of its batched runs
 * (SOS_ETIMEOUT after a lookback wait ran out of time). */
sos_status sos_batch_sync_status(int device);

/*
 * Continue filtering from the filter's resident device state (a [K][2]
 * float32 array kept on the device between calls) and update it in place, so
 * that consecutive chunks equal one long call.  Calls on one filter must be
 * serialized on one stream.
 */
sos_status sos_filter_stream_push(sos_filter *f, const float *x_dev, float *y_dev, int64_t n, void *stream);

/*
 * Read and/or replace the resident state.
 *   z_out  [K][2] float32 receives the state (NULL = skip)
 *   z_in   [K][2] float32 new state (NULL = keep)
 *   on_device  nonzero: z_out/z_in are device pointers and the copies are
 *              enqueued on the filter's last stream; zero: host pointers and
 *              the call synchronizes that stream first.
 * Returns the sticky device status (SOS_ETIMEOUT after a lookback timeout).
 */
sos_status sos_filter_stream_state(sos_filter *f, float *z_out, const float *z_in, int on_device);

/*
 * Synchronize the filter's last stream and return the sticky device status.  SOS_ETIMEOUT means
 * that a device wait (a lookback or barrier wait) ran past sos_tuning.spin_budget_cycles: the
 * kernel recorded it and returned early, so the outputs and final states of the runs issued since
 * then are undefined.  Reporting it clears it: the call then resets the filter's status word and
 * ticket counter, so that the runs issued after it are valid again.
 */
sos_status sos_filter_sync_status(sos_filter *f);

/*
 * Phase trace for diagnostics (no counterpart in the paper's method; it
 * measures where a tile's time goes).  When buf_dev is non-NULL, every
 * following launch on this filter writes 32 uint64 words per work item at
 * buf_dev[32 * i ...] for items i < capacity_blocks; times are the device
 * global timer in ns.  The items and slots depend on the kernel:
 *   PH solver (per tile): [0] tile + 1; coordinator: [1] lookback start,
 *     [2] incoming state resolved, [3] group states posted; first compute warp:
 *     [4] iteration start, [5] next ticket known, [6] particular pass done,
 *     [7] lane scan done, [8] fold done, [9] correction start, [10] group state
 *     observed, [11] row states stored, [12] stored, [14]/[15] input stash;
 *     [13] SM id.
 *   PH on the tensor cores (per tile): [0] tile + 1, [13] SM id; coordinator: [1]
 *     start, [26] predecessors' local carries observed, [27] anchor carries
 *     observed, [2] incoming state resolved, [3] group states posted; producer: [16]
 *     ticket drawn, [17] loads issued; MMA issuer: [18] first products issued,
 *     [19] remainder products issued, [20] correction issued; [21] input
 *     remainder formed; epilogue (first warp of each warpgroup): [4]/[22]
 *     accumulator observed, [7]/[23] lane scan done, [8] fold start, [28] tile
 *     carry folded (the folding warp), [9]
 *     correction start, [10] group state observed, [11] state operand posted,
 *     [12]/[24] correction observed, [14]/[25] outputs stored.
 *   cyclic reduction, cascade carry (per tile): see the kernel's source.
 *   cyclic reduction, per-section carries (per ticket): [0] ticket + 1,
 *     [1] start, [2] after drawing the ticket, [3] after stage-in, [4 + 3s]
 *     block carry of section s published, [5 + 3s] incoming state of section s
 *     known, [6 + 3s] lookback rounds (low 32 bits) and waits (high 32 bits),
 *     [28] before stage-out, [29] end, [30] SM id.
 * buf_dev = NULL switches it off.  The caller owns the buffer.  Errors:
 * SOS_EINVAL for capacity < 0.
 */
sos_status sos_filter_trace(sos_filter *f, uint64_t *buf_dev, int64_t capacity_blocks);

/*
 * sos_filter_run_noalloc: the same filtering, for callers that cannot allocate device memory
 * while they filter.  (The paper has no counterpart; this is a library service.)  A real-time
 * thread, such as an audio or radio receive loop, must not call cudaMalloc or cudaFree in its
 * processing loop, because those calls can block and synchronize the device; other applications
 * hand out all device memory at start-up.  Such a caller creates the filter (sos_filter_create
 * allocates its tables once, including the final-state tables for every length) and then filters
 * with this entry point, which allocates nothing: no cudaMalloc, cudaFree or other allocating
 * CUDA routine, and no host heap allocation.  The scratch memory of a run (lookback descriptors
 * and ticket counter) lives in one fixed array of 4.6 MiB in the library's device code, which
 * every GPU that loads the library holds until the process exits.
 *   Arguments and results are those of sos_filter_run with the PH solver at N = 64 (the default
 *   solver), and so are its outputs and final states, bit for bit.
 *   n            at most SOS_NOALLOC_MAX_SAMPLES samples per call, else SOS_EBUDGET
 *   The first call on a device looks up the array's device address on the current device
 *   (a one-time set-up).
 *   All calls on a device share the array and keep its last contents: each pass first clears the
 *   ticket counter and the descriptors it will use (with cudaMemsetAsync on `stream`), so nothing
 *   needs clearing by the caller, but calls that overlap on the GPU (different streams, or
 *   different host threads without ordering) race and must be serialized by the caller.
 */
#define SOS_NOALLOC_MAX_SAMPLES (1LL << 28)
sos_status sos_filter_run_noalloc(sos_filter *f, const float *x_dev, float *y_dev, int64_t n,
                                  const float *zi_dev, float *zf_dev, void *stream);

/*
 * Serving: a request loop with continuous batching over many streams (a
 * library service built on sos_filter_run_batch_ex; the paper's method is the
 * per-batch filtering).  Every stream is a cascade whose [K][2] state stays on
 * the device between chunks, so a stream's next chunk continues from its last
 * one with no host round trip.  Requests name caller-owned device buffers; a
 * scheduler thread admits the oldest ready chunks (at most one chunk of a
 * stream in flight, chunks of a stream in submission order) while the bytes in
 * flight (8 per sample, 4 in place) stay within the budget, issues each batch
 * on one of `max_inflight` CUDA streams so that batches overlap on the device,
 * and records completions from a host function behind each batch.  Requests
 * that arrive while others are on the device join the next batch as soon as
 * budget and a batch slot free up.
 */
typedef struct sos_server sos_server;

typedef struct {
    int64_t budget_bytes; /* device bytes of chunks in flight; 0 = 16 GiB */
    int max_batch;        /* chunks per batch; 0 = 4096 */
    int max_inflight;     /* batches in flight on the device (1..8); 0 = 4 */
} sos_server_config;

typedef struct {
    uint64_t request_id;
    int stream_id;
    int status;        /* sos_status of the request */
    int64_t n;         /* samples */
    double t_submit;   /* host steady-clock seconds: submission (or scheduled arrival, replay) */
    double t_start;    /* admitted into a batch */
    double t_done;     /* completion observed (host function behind the batch) */
} sos_completion;

typedef struct {
    int64_t submitted, completed, rejected, batches, max_batch_seen, samples_done, inflight_bytes;
} sos_server_stats;

/* Create a server on the current device (NULL cfg = defaults). */
sos_status sos_server_create(const sos_server_config *cfg, sos_server **out);
/* Finish every queued request, then release the server, its streams and their states. */
sos_status sos_server_destroy(sos_server *s);
/* Add a stream: K sections `sos` [K][5] (as sos_filter_create), initial state zi [K][2] (host,
 * NULL = zeros); *stream_id receives its index.  Allocates device memory. */
sos_status sos_server_add_stream(sos_server *s, int n_sections, const double *sos, const float *zi, int *stream_id);
/* Queue chunk x_dev[n] -> y_dev[n] (device buffers, may be equal; they must stay valid until the
 * request completes) for a stream.  Errors: SOS_EINVAL, SOS_EBUDGET (chunk larger than the budget). */
sos_status sos_server_submit(sos_server *s, int stream_id, const float *x_dev, float *y_dev, int64_t n,
                             uint64_t *request_id);
/* Move up to `max` completions to out (oldest first), waiting up to wait_ms for one if none is
 * ready.  Returns the first error of any batch (sticky) or SOS_OK.  The requests of a batch that
 * could not be issued complete with its error, and their streams keep the state they had before
 * it (the next chunk continues as if the failed one had been skipped). */
sos_status sos_server_poll(sos_server *s, sos_completion *out, int max, int *n_out, int wait_ms);
/* Wait until every queued request has completed. */
sos_status sos_server_drain(sos_server *s);
/* Copy a stream's resident state [K][2] to the host after its queued chunks have completed. */
sos_status sos_server_stream_state(sos_server *s, int stream_id, float *z_host);
sos_status sos_server_get_stats(sos_server *s, sos_server_stats *out);
/*
 * Load replay for measurements: request i (stream stream_ids[i], buffers x_dev[i] -> y_dev[i],
 * n[i] samples) arrives t_arrival[i] seconds after the call (non-decreasing); latency[i] receives
 * its completion time minus its scheduled arrival.  Returns when all have completed.  The caller
 * must not submit or poll on the server meanwhile (the replay consumes the completion queue).
 * Errors, found before any request is queued: SOS_EINVAL (NULL arrays or buffers, a bad stream id,
 * n[i] <= 0), SOS_EBUDGET (a chunk larger than the budget).
 */
sos_status sos_server_replay(sos_server *s, int64_t n_req, const int32_t *stream_ids, const float *const *x_dev,
                             float *const *y_dev, const int64_t *n, const double *t_arrival, double *latency);

/*
 * Autotuner: on the current device, time each candidate launch configuration
 * -- divide-and-conquer cyclic reduction with the cascade carry at N = 32 (8
 * groups per tile) or N = 64 (4 groups per tile), PH factorization at N = 64
 * with 7 or 10 groups per tile, double-thread-group cyclic reduction at N = 64
 * (4 groups of two warps per tile) and PH factorization on the tensor cores (8
 * groups per tile); L = 32 threads per group (thread group)
 * throughout -- for 1 to 8 sections and lengths 2^16, 2^20, 2^24 and 2^28 (up to
 * 2^max_log2n, 0 = 28), and keep the fastest per (section count, length).
 * Afterwards every run of a filter created with default tuning (all fields 0)
 * uses the choice for its section count and the nearest length.  Synchronous;
 * allocates and frees 2^(max_log2n + 3) bytes of device memory; a second or two.
 *   report  NULL, or host float[8][4][6] receiving the measured GS/s
 *           (sections, length 2^16..2^28, candidate CR32/CR64/PH/DTCR/PH with
 *           10 groups per tile/PH on the tensor cores)
 */
sos_status sos_autotune(int max_log2n, float *report);

/* The autotuned choice for K sections and n samples on the current device:
 * solver (SOS_SOLVER_CR / SOS_SOLVER_PH / SOS_SOLVER_DTCR / SOS_SOLVER_TC) and N; both
 * 0 if no autotuning ran. */
sos_status sos_autotune_choice(int n_sections, int64_t n, int *solver, int *N);
/* The same with the groups per tile of a PH choice (7 or 10; 8 for SOS_SOLVER_TC; 0 for the
 * other solvers) in *groups_per_cta (may be NULL). */
sos_status sos_autotune_choice_ex(int n_sections, int64_t n, int *solver, int *N, int *groups_per_cta);

/*
 * Autotuner of batched runs (Sec. IV-D configurations for many signals): on
 * the current device, time the batch kernel's two tile geometries (N = 64 and
 * N = 32 samples per thread, 7 groups of L = 32 threads per tile) for 1 to 8
 * sections on batches of 2^24 samples in equal signals of 2^12, 2^15, 2^18 and
 * 2^21 samples, and keep the faster per (section count, length).  Afterwards
 * every batched run (sos_filter_run_batch[_ex], sos_batch_plan_create, the
 * serving loop) takes the choice for each signal whose filter's tuning leaves
 * N at 0.  Synchronous; allocates and frees 128 MiB of device memory.
 *   report  NULL, or host float[8][4][2] receiving the measured GS/s
 *           (sections, signal length 2^12..2^21, geometry N = 64 / N = 32)
 */
sos_status sos_autotune_batch(float *report);

/* The batch autotuner's samples per thread for a signal of K sections and n
 * samples on the current device (64 or 32); 0 if sos_autotune_batch has not run. */
sos_status sos_autotune_batch_choice(int n_sections, int64_t n, int *N);

/* Human-readable name of a status code (static storage). */
const char *sos_status_string(sos_status s);

#ifdef __cplusplus
}
#endif
#endif /* SOSFILT_H */
