// Host stand-ins below the library's host code (sosfilt_api.cpp) for tests without a GPU: the CUDA
// runtime (host memory, streams that run their work at once) and the kernel launchers.  Test
// infrastructure only.
//
// A launcher records its launch (which kernel, K, N, b0 handling, grid, and a copy of its parameter
// block) and applies a marker in place of the filter: every output sample is twice its input, and
// word 0 of the final state is word 0 of the initial state plus the samples processed (the other
// words are copied).  So a test can tell that every sample went through exactly one launch per pass
// and that states were chained, and can read the tables the host built from the recorded
// parameters (their pointers are host memory here).  Events measure simulated time: the sum of a
// per-(kernel, N, K) cost over the launches recorded between them, so that the autotuner's choice
// can be steered.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <set>
#include <vector>

#include "cuda_runtime.h"
#include "sosfilt.h"
#include "sosfilt_internal.h"

struct host_stream {
    int id;
};
struct host_event {
    size_t mark;  // launches recorded before the event
};

namespace {
struct Launch {
    int kind, K, N, norm;
    long long grid;
    std::vector<unsigned char> params;
};
std::vector<Launch> g_launches;
bool g_light = false;          // record no parameter blocks and skip the marker (timing runs)
float g_cost[7][3][9] = {};    // simulated time of a launch, ms, by kind, N (32, 64, 128) and K

int n_index(int N) { return N == 32 ? 0 : N == 64 ? 1 : 2; }

bool g_recording = false;  // the recorder's own allocations are not the library's

template <class P>
void record(int kind, int K, int N, bool norm, long long grid, const P &p) {
    g_recording = true;
    struct Done {
        ~Done() { g_recording = false; }
    } done;
    Launch l{kind, K, N, norm ? 1 : 0, grid, {}};
    if (!g_light) {
        l.params.resize(sizeof(P));
        std::memcpy(l.params.data(), &p, sizeof(P));
    }
    g_launches.push_back(std::move(l));
}

void mark(const float *x, float *y, long long n, const float *zi, float *zf, int K) {
    if (g_light) return;
    for (long long i = 0; i < n; ++i) y[i] = 2.0f * x[i];
    if (zf)
        for (int j = 0; j < 2 * K; ++j) zf[j] = (zi ? zi[j] : 0.0f) + (j == 0 ? static_cast<float>(n) : 0.0f);
}
}  // namespace

cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int *d) {
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaDeviceSynchronize(void) { return cudaSuccess; }
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr, int) {
    *v = 4;  // a small "GPU": four SMs
    return cudaSuccess;
}
// calls of the allocating runtime routines (cudaMalloc, cudaMallocHost, cudaFree, cudaFreeHost)
long long g_runtime_allocs = 0;
cudaError_t cudaMalloc(void **p, size_t bytes) {
    ++g_runtime_allocs;
    *p = std::calloc(1, bytes ? bytes : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p) {
    ++g_runtime_allocs;
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaMallocHost(void **p, size_t bytes) { return cudaMalloc(p, bytes); }
cudaError_t cudaFreeHost(void *p) { return cudaFree(p); }
// host memory is its own device mapping here; address 16 stands for memory without a mapping
cudaError_t cudaHostGetDevicePointer(void **dptr, void *hptr, unsigned) {
    if (reinterpret_cast<uintptr_t>(hptr) == 16) return cudaErrorInvalidValue;
    *dptr = hptr;
    return cudaSuccess;
}
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind) {
    std::memmove(dst, src, bytes);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind k, cudaStream_t) {
    return cudaMemcpy(dst, src, bytes, k);
}
cudaError_t cudaMemset(void *dst, int v, size_t bytes) {
    std::memset(dst, v, bytes);
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void *dst, int v, size_t bytes, cudaStream_t) { return cudaMemset(dst, v, bytes); }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) {
    *s = new host_stream{0};
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
bool g_capturing = false;  // host_set_capturing: every stream reports an active capture
cudaError_t cudaStreamIsCapturing(cudaStream_t, cudaStreamCaptureStatus *st) {
    *st = g_capturing ? cudaStreamCaptureStatusActive : cudaStreamCaptureStatusNone;
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) {
    delete s;
    return cudaSuccess;
}
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t *e) {
    *e = new host_event{0};
    return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned) { return cudaEventCreate(e); }
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t) {
    e->mark = g_launches.size();
    return cudaSuccess;
}
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t e) {
    delete e;
    return cudaSuccess;
}
// the simulated times of the launches recorded between the two events (1 ms each by default)
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b) {
    double t = 0.0;
    for (size_t i = a->mark; i < b->mark && i < g_launches.size(); ++i) {
        const Launch &l = g_launches[i];
        const float c = g_cost[l.kind][n_index(l.N)][l.K];
        t += c > 0.f ? c : 1.0;
    }
    *ms = static_cast<float>(t);
    return cudaSuccess;
}

namespace sosk {

sos_status run_lane_scratch(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf,
                            cudaStream_t s, const Scratch &sc, unsigned (*next_epoch)(int, cudaStream_t));

bool dccr_available(int, int, bool, int) { return true; }
int cascade_blocks_per_sm_32(int, bool) { return 1; }
int cascade_blocks_per_sm_64(int, bool) { return 1; }
size_t cascade_smem_32(int) { return 0; }
size_t cascade_smem_64(int) { return 0; }
int lane_blocks_per_sm_n32a(int, bool) { return 2; }
int lane_blocks_per_sm_n32b(int, bool) { return 2; }
int lane_blocks_per_sm_n64a(int, bool) { return 1; }
int lane_blocks_per_sm_n64b(int, bool) { return 1; }
int lane_blocks_per_sm_n64w10a(int, bool) { return 1; }
int lane_blocks_per_sm_n64w10b(int, bool) { return 1; }
int batch_all_blocks_per_sm() { return 1; }
int dtcr_blocks_per_sm(int, bool) { return 1; }
int tc_blocks_per_sm(int) { return 1; }
int default_lbm(int N) { return N <= 32 ? 4 : N == 64 ? 2 : 1; }

cudaError_t launch_dccr(int K, int N, bool norm, int, const PassParams &p, long long grid, cudaStream_t) {
    record(4, K, N, norm, grid, p);
    mark(p.x, p.y, p.n, p.zi, p.zf, K);
    return cudaSuccess;
}

#define HOST_LANE(K, N, W)                                                                             \
    template <>                                                                                        \
    cudaError_t launch_lane<K, N, W>(bool norm, const LaneParams<K> &p, long long grid, cudaStream_t) {  \
        record(1, K, N, norm, grid, p);                                                                \
        mark(p.x, p.y, p.n, p.zi, p.zf, K);                                                            \
        return cudaSuccess;                                                                            \
    }
#define HOST_CAS(K, N)                                                                                \
    template <>                                                                                       \
    cudaError_t launch_cascade<K, N>(bool norm, const CasParams<K, N> &p, long long grid, cudaStream_t) { \
        record(2, K, N, norm, grid, p);                                                               \
        mark(p.x, p.y, p.n, p.zi, p.zf, K);                                                           \
        return cudaSuccess;                                                                           \
    }
// The single batch kernel: counted, and recorded as one launch record per class it covers (the
// class's queue in the layout of BatchParams, so the tests read every class alike; N = the class's
// samples per lane).
long long g_batch_all_launches = 0;
cudaError_t launch_batch_all(const BatchAllParams &p, long long grid, cudaStream_t) {
    ++g_batch_all_launches;
    for (int i = 0; i < p.n_classes; ++i) {
        const BatchQueue &q = p.q[i];
        const BatchParams<1> bp{q.sigs, q.tile_sig, q.n_tiles, q.desc, q.ticket, q.ticket_base, q.epoch, p.status,
                                p.spin_budget};
        const int K = batch_class_k(p.code[i]);
        record(3, K, batch_geom_n(batch_class_geom(p.code[i])), (p.code[i] & 1) != 0, grid, bp);
        if (g_light) continue;
        std::set<int> sigs(q.tile_sig, q.tile_sig + q.n_tiles);
        for (int j : sigs) {
            const BatchSig &g = q.sigs[j];
            mark(g.x, g.y, g.n, g.zi, g.zf, K);
        }
    }
    return cudaSuccess;
}

#define HOST_DTCR(K)                                                                                \
    template <>                                                                                     \
    cudaError_t launch_dtcr<K>(bool norm, const CasParams<K, 64> &p, long long grid, cudaStream_t) { \
        record(5, K, 64, norm, grid, p);                                                            \
        mark(p.x, p.y, p.n, p.zi, p.zf, K);                                                         \
        return cudaSuccess;                                                                         \
    }
// the tensor-core kernel: recorded as kind 6; its operand image and final-state table must exist
#define HOST_TC(K)                                                                                           \
    template <>                                                                                              \
    cudaError_t launch_tc<K>(const LaneParams<K> &p, const float *img, const float *gtail, long long grid, \
                             cudaStream_t) {                                                                 \
        if (!img || !gtail) return cudaErrorInvalidValue;                                                    \
        record(6, K, 64, false, grid, p);                                                                    \
        mark(p.x, p.y, p.n, p.zi, p.zf, K);                                                                  \
        return cudaSuccess;                                                                                  \
    }
#define HOST_ALL(K) HOST_LANE(K, 32, 7) HOST_LANE(K, 64, 7) HOST_LANE(K, 64, 10) HOST_CAS(K, 32) HOST_CAS(K, 64) \
    HOST_DTCR(K) HOST_TC(K)
HOST_ALL(1) HOST_ALL(2) HOST_ALL(3) HOST_ALL(4) HOST_ALL(5) HOST_ALL(6) HOST_ALL(7) HOST_ALL(8)

}  // namespace sosk

namespace {
unsigned g_epoch = 0;
unsigned scratch_epoch(int, cudaStream_t) { return ++g_epoch; }
// global operator new calls (the harness is linked with -Bsymbolic, so the library's own calls
// bind here)
long long g_heap_allocs = 0;
}  // namespace

void *operator new(size_t bytes) {
    if (!g_recording) ++g_heap_allocs;
    void *p = std::malloc(bytes ? bytes : 1);
    if (!p) throw std::bad_alloc();
    return p;
}
void operator delete(void *p) noexcept { std::free(p); }
void operator delete(void *p, size_t) noexcept { std::free(p); }

// Test hooks.
extern "C" {
// a run with caller-provided lookback scratch of desc_words words, filled with a non-zero pattern
// beforehand (the path of sos_filter_run_noalloc).  where[0..1]: the scratch addresses used;
// where[2]: the ticket counter afterwards; where[3], where[4]: calls of allocating runtime routines
// and of operator new during the run; where[5]: the words of the scratch that are still non-zero
// afterwards (descriptors the run neither cleared nor wrote).
int host_run_scratch(sos_filter *f, const float *x, float *y, long long n, const float *zi, float *zf,
                     long long desc_words, unsigned long long *where) {
    std::vector<unsigned long long> desc(static_cast<size_t>(desc_words) + 1, 0xabababababababULL), ticket(1, 12345);
    sosk::Scratch sc{desc.data(), static_cast<size_t>(desc_words), ticket.data()};
    where[0] = reinterpret_cast<unsigned long long>(desc.data());
    where[1] = reinterpret_cast<unsigned long long>(ticket.data());
    const long long rt0 = g_runtime_allocs, heap0 = g_heap_allocs;
    const int rc = sosk::run_lane_scratch(f, x, y, n, zi, zf, nullptr, sc, scratch_epoch);
    where[3] = static_cast<unsigned long long>(g_runtime_allocs - rt0);
    where[4] = static_cast<unsigned long long>(g_heap_allocs - heap0);
    where[2] = ticket[0];
    unsigned long long left = 0;
    for (size_t i = 0; i < static_cast<size_t>(desc_words); ++i) left += desc[i] != 0;
    where[5] = left;
    return rc;
}
void host_reset(void) { g_launches.clear(); }
void host_set_light(int on) { g_light = on != 0; }
void host_set_capturing(int on) { g_capturing = on != 0; }
void host_set_cost(int kind, int N, int K, float ms) { g_cost[kind][n_index(N)][K] = ms; }
int host_launches(void) { return static_cast<int>(g_launches.size()); }
// single-kernel batch launches so far
long long host_batch_all_launches(void) { return sosk::g_batch_all_launches; }
// kind (1 PH lane, 2 cyclic-reduction cascade, 3 batch, 4 per-section cyclic reduction, 5 double-
// thread-group cyclic reduction), K, N,
// b0 normalization, grid; returns the parameter block's size and copies up to cap bytes of it
long long host_launch(int i, int *info, long long *grid, void *params, long long cap) {
    const Launch &l = g_launches.at(static_cast<size_t>(i));
    info[0] = l.kind;
    info[1] = l.K;
    info[2] = l.N;
    info[3] = l.norm;
    *grid = l.grid;
    const long long n = static_cast<long long>(l.params.size());
    if (params) std::memcpy(params, l.params.data(), static_cast<size_t>(n < cap ? n : cap));
    return n;
}
// byte offsets in LaneParams<K>: x, y, n, G, n_tiles, zi, zf, gain, m_last, tab, sec, MX, A_tail,
// desc, ticket, ticket_base, epoch, spin_budget, trace, trace_tiles, aligned
#define LANE_OFFS(K)                                                                                          \
    case K: {                                                                                                 \
        using P = sosk::LaneParams<K>;                                                                        \
        const long long o[] = {offsetof(P, x),    offsetof(P, y),   offsetof(P, n),  offsetof(P, G),          \
                               offsetof(P, n_tiles), offsetof(P, zi), offsetof(P, zf), offsetof(P, gain),     \
                               offsetof(P, m_last), offsetof(P, tab), offsetof(P, sec), offsetof(P, MX),      \
                               offsetof(P, A_tail), offsetof(P, desc), offsetof(P, ticket),                   \
                               offsetof(P, ticket_base), offsetof(P, epoch), offsetof(P, spin_budget),        \
                               offsetof(P, trace), offsetof(P, trace_tiles), offsetof(P, aligned)};           \
        std::memcpy(out, o, sizeof o);                                                                        \
        return static_cast<long long>(sizeof(P));                                                             \
    }
long long host_lane_layout(int K, long long *out) {
    switch (K) {
        LANE_OFFS(1) LANE_OFFS(2) LANE_OFFS(3) LANE_OFFS(4) LANE_OFFS(5) LANE_OFFS(6) LANE_OFFS(7) LANE_OFFS(8)
        default: return -1;
    }
}
// byte offsets in CasParams<K, N>: n, G, n_tiles, gain, tab, sec, H, A_tail; returns its size
#define CAS_OFFS(K, N)                                                                                   \
    if (k == K && n == N) {                                                                              \
        using P = sosk::CasParams<K, N>;                                                                 \
        const long long o[] = {offsetof(P, n),   offsetof(P, G),   offsetof(P, n_tiles), offsetof(P, gain), \
                               offsetof(P, tab), offsetof(P, sec), offsetof(P, H),       offsetof(P, A_tail)}; \
        std::memcpy(out, o, sizeof o);                                                                   \
        return static_cast<long long>(sizeof(P));                                                        \
    }
long long host_cas_layout(int k, int n, long long *out) {
    CAS_OFFS(1, 32) CAS_OFFS(2, 32) CAS_OFFS(5, 32) CAS_OFFS(8, 32)
    CAS_OFFS(1, 64) CAS_OFFS(2, 64) CAS_OFFS(5, 64) CAS_OFFS(8, 64)
    return -1;
}
// sizeof(SecCoef) and the byte offsets in SecCoef: t0, b1, ne, f, nf, qo, qe, tn, tc, zscale; in
// PassParams: sec, lane_pow, grp_pow, cta_pow, n_sec, gain, n
void host_pass_layout(long long *out) {
    using S = sosk::SecCoef;
    using P = sosk::PassParams;
    const long long o[] = {sizeof(S), offsetof(S, t0), offsetof(S, b1), offsetof(S, ne), offsetof(S, f),
                           offsetof(S, nf), offsetof(S, qo), offsetof(S, qe), offsetof(S, tn), offsetof(S, tc),
                           offsetof(S, zscale), offsetof(P, sec), offsetof(P, lane_pow), offsetof(P, grp_pow),
                           offsetof(P, cta_pow), offsetof(P, n_sec), offsetof(P, gain), offsetof(P, n)};
    std::memcpy(out, o, sizeof o);
}
// sizeof(LaneSec), sizeof(BatchSig) and the byte offsets in BatchSig: x, y, n, G, tile0, zi, zf,
// tab, gain; in BatchParams<1>: sigs, tile_sig, n_tiles; in BatchSig: sec, MX, Mm
void host_batch_layout(long long *out) {
    using B = sosk::BatchSig;
    using P = sosk::BatchParams<1>;
    const long long o[] = {sizeof(sosk::LaneSec), sizeof(B), offsetof(B, x), offsetof(B, y), offsetof(B, n),
                           offsetof(B, G), offsetof(B, tile0), offsetof(B, zi), offsetof(B, zf), offsetof(B, tab),
                           offsetof(B, gain), offsetof(P, sigs), offsetof(P, tile_sig), offsetof(P, n_tiles),
                           offsetof(B, sec), offsetof(B, MX), offsetof(B, Mm)};
    std::memcpy(out, o, sizeof o);
}
}
