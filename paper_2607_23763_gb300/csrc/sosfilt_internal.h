// Internal structures shared by the host side (sosfilt_api.cpp) and the
// kernels (sosfilt_dccr.cuh).  Not part of the public ABI.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace sosk {

constexpr int kL = 32;        // threads per group: one warp, every lane-scan round is a shuffle
constexpr int kMaxD = 7;      // log2 of the largest supported N (128)
constexpr int kMaxPass = 8;   // sections filtered per kernel launch (one pass)
constexpr int kWarps = 4;     // groups (warps) per thread block

// Group-transition table per section: (T^C)^k for k = 0..32, then (T^C)^(32 i) for i = 0..16.
constexpr int kPow32 = 33;
constexpr int kMaxLBM = 16;
constexpr int kGrpPowStride = kPow32 + kMaxLBM + 1;

// Phase trace (diagnostics): per thread block kTraceSlots 64-bit words, indexed by ticket.
//   [0] ticket + 1   [1] start   [2] after the ticket   [3] after stage-in
//   [4 + 3s] block carry published (after the first barrier of section s)
//   [5 + 3s] incoming state known (after the second barrier of section s)
//   [6 + 3s] lookback rounds (low 32 bits) and waits (high 32 bits) of section s
//   [28] before stage-out   [29] end   [30] SM id
constexpr int kTraceSlots = 32;
// Phase trace of the cascade kernel, per tile: [0] tile + 1, coordinator: [1] stash observed,
// [2] tile carry folded, [3] incoming state resolved, [4] group states posted, [5] lookback
// windows (low 32 bits) and waits (high 32 bits); warp 0: [6] pass start, [7] pass end,
// [8] before waiting for the group state, [9] group state observed, [10] output issued; [11] SM id.

// Device status bits (sticky, OR-ed by the kernels).
constexpr int kDevErrTimeout = 1;

// Per-section tables, float32, derived in float64 on the host for one N.
// Level i of the reduction holds y[m] + e_i y[m - 2^i] + f_i y[m - 2^(i+1)] = v_i[m].
struct SecCoef {
    // the same coefficients duplicated into (even, odd) pairs for packed f32x2 FMAs on the two
    // divide-and-conquer chains
    float2 p_t0, p_t1, p_t2, p_t3, p_t4;
    float2 p_ne[kMaxD + 1], p_f[kMaxD + 1], p_nf[kMaxD + 1];
    float2 p_q0[kMaxD + 1];         // (qe[i][0], qo[i][0]): state injection, z1 part
    float2 p_q1[kMaxD + 1];         // (qe[i][1], qo[i][1]): state injection, z2 part
    float t0, t1, t2, t3, t4;       // first-level taps of B(z) A(-z) (Eq. 23 when b0 = 1)
    float b1, b2, a1, a2;           // section coefficients used by the terminal state (b / b0 when normalized)
    float ne[kMaxD + 1];            // -e_i, i = 1..D-1
    float f[kMaxD + 1];             // +f_i, i = 1..D-1
    float nf[kMaxD + 1];            // -f_i, i = 1..D-1
    float qo[kMaxD + 1][2];         // state injection at the first odd-chain row of level i = 1..D
    float qe[kMaxD + 1][2];         // state injection at the first even-chain row of level i = 1..D
    float tn[5][4];                 // (T^N)^(2^k), k = 0..4, row-major 2x2, T = [[-a1, 1], [-a2, 0]]
    float tc[kWarps + 1][4];        // (T^C)^w, w = 0..kWarps: composition inside a thread block
    float zscale, zscale_inv;       // carried state = zscale * true state (b0 normalization)
};

struct PassParams {
    const float *x;
    float *y;
    long long n;       // samples in the signal
    long long G;       // groups = ceil(n / C)
    const float *zi;   // device [kMaxPass][2] of this pass (true domain) or nullptr
    float *zf;         // device [kMaxPass][2] of this pass or nullptr
    float gain;        // input multiplier (product of all b0 when normalized; first pass only, else 1)
    unsigned long long *desc;   // lookback descriptors [kMaxPass][blocks][2] 64-bit words
    unsigned long long *ticket; // monotone ticket counter of the filter object
    unsigned long long ticket_base;
    unsigned int epoch;         // 30-bit launch tag, never 0
    const float4 *lane_pow;     // [kMaxPass][32]: (T^N)^l
    const float4 *grp_pow;      // [kMaxPass][kGrpPowStride]: (T^C)^k, k = 0..32; (T^C)^(32 i), i = 0..16
    const float4 *cta_pow;      // same layout for the block transition S = T^(kWarps C)
    int *status;
    long long spin_budget;      // cycles
    int aligned;                // x and y are 16-byte aligned
    int n_sec;                  // sections in this pass (== template K)
    unsigned long long *trace;  // nullptr, or [blocks][kTraceSlots] phase trace
    long long trace_blocks;     // capacity of trace in blocks
    SecCoef sec[kMaxPass];
};

// ---- persistent kernel with one carry per tile for the whole cascade (sosfilt_cascade.cuh)
constexpr int kMaxWin = 16;  // lookback windows of 32 tiles

template <int K, int N>
struct CasParams {
    const float *x;
    float *y;
    long long n, G, n_tiles;    // samples, groups, tiles (W groups each)
    const float *zi;            // device [K][2] initial state of this pass (true domain) or nullptr
    float *zf;                  // device [K][2] final state of this pass or nullptr
    float gain;                 // input multiplier (product of all b0 when normalized; first pass only)
    unsigned long long *desc;   // [n_tiles][2K] tagged carry words
    unsigned long long *ticket;
    unsigned long long ticket_base;
    unsigned int epoch;
    int *status;
    long long spin_budget;
    int aligned;                // x and y 16-byte aligned
    const float *tab;           // (M_N)^lane, (A_T)^lane [32][MS] packed; A_C, A_T, (A_T)^(32 w) (w = 1..kMaxWin) dense
    unsigned long long *trace;  // nullptr, or [n_tiles][kTraceSlots] phase trace (see kCasTrace*)
    long long trace_tiles;
    SecCoef sec[K];
    alignas(8) float H[2 * K][N];        // output at lane sample m of the zero-input cascade from unit state j
    float A_tail[2 * K * (K + 1)];  // cascade transition over the last group's real samples (packed)
};

// Launch one pass of the cascade kernel (explicit specializations in sosfilt_cascade_n*.cu).
template <int K, int N>
cudaError_t launch_cascade(bool norm, const CasParams<K, N> &p, long long grid, cudaStream_t s);
#define SOSK_DECLARE_CASCADE(K, N) \
    template <>                    \
    cudaError_t launch_cascade<K, N>(bool norm, const CasParams<K, N> &p, long long grid, cudaStream_t s);
#define SOSK_DECLARE_CASCADE_N(N)                                                                    \
    SOSK_DECLARE_CASCADE(1, N) SOSK_DECLARE_CASCADE(2, N) SOSK_DECLARE_CASCADE(3, N)                 \
    SOSK_DECLARE_CASCADE(4, N) SOSK_DECLARE_CASCADE(5, N) SOSK_DECLARE_CASCADE(6, N)                 \
    SOSK_DECLARE_CASCADE(7, N) SOSK_DECLARE_CASCADE(8, N)
SOSK_DECLARE_CASCADE_N(32)
SOSK_DECLARE_CASCADE_N(64)
// Thread blocks of the cascade kernel that fit on one SM (0 if unavailable).
int cascade_blocks_per_sm(int K, int N, bool norm);

// ---- double-thread-group cyclic reduction (sosfilt_dtcr.cuh): the cascade-carry kernel with two
// warps per group (one per parity), on the N = 64 cyclic-reduction tables (tiles of 4 groups)
template <int K>
cudaError_t launch_dtcr(bool norm, const CasParams<K, 64> &p, long long grid, cudaStream_t s);
#define SOSK_DECLARE_DTCR(K) \
    template <>              \
    cudaError_t launch_dtcr<K>(bool norm, const CasParams<K, 64> &p, long long grid, cudaStream_t s);
SOSK_DECLARE_DTCR(1) SOSK_DECLARE_DTCR(2) SOSK_DECLARE_DTCR(3) SOSK_DECLARE_DTCR(4)
SOSK_DECLARE_DTCR(5) SOSK_DECLARE_DTCR(6) SOSK_DECLARE_DTCR(7) SOSK_DECLARE_DTCR(8)
int dtcr_blocks_per_sm(int K, bool norm);
int cascade_warps(int N);       // compute warps (groups) per block
size_t cascade_smem(int K, int N);

// ---- PH-factorization kernel with a skewed direct-form-II particular pass (sosfilt_lane.cuh)
constexpr int kLaneW = 7;    // compute warps per block, one group each; a tile is kLaneW groups
constexpr int kLaneWide = 10;  // the wide variant at N = 64: 10 groups per tile (sos_tuning.groups_per_cta)

// Per-section constants of the skewed-pass kernel, in the kernel's domain (b / b0 and b0 = 1 when
// normalized; carried state = zscale * true state).
struct LaneSec {
    float4 c;      // b1, b2, -a1, -a2
    float4 tn[5];  // (T^N)^(2^r), r = 0..4, row-major 2x2, T the section's one-sample transition
    float b0, zscale, zscale_inv, pad;
};

template <int K>
struct LaneParams {
    const float *x;
    float *y;
    long long n, G, n_tiles;    // samples, groups of 32 N samples, tiles of kLaneW groups
    const float *zi;            // device [K][2] initial state of this pass (true domain) or nullptr
    float *zf;                  // device [K][2] final state of this pass or nullptr
    float gain;                 // input multiplier (product of all b0 when normalized; first pass only)
    unsigned long long *desc;   // [n_tiles][2][2K] tagged carry words: local, resolved
    unsigned long long *ticket;
    unsigned long long ticket_base;
    unsigned int epoch;
    int *status;
    long long spin_budget;
    int aligned;                // x and y 16-byte aligned
    int m_last;                 // position of the signal's last sample inside its lane
    const float *tab;           // global table block, layout LaneDims<K, N>
    unsigned long long *trace;  // nullptr, or [n_tiles][kTraceSlots] phase trace (kLaneTrace*)
    long long trace_tiles;
    LaneSec sec[K];
    // blocks (k, j), j < k, of the lane transition M_N, row-major 2x2 at k (k - 1) / 2 + j
    float4 MX[K > 1 ? K * (K - 1) / 2 : 1];
    float A_tail[2 * K * (K + 1)];  // packed cascade transition over m_last + 1 samples
};

// Phase trace of the skewed-pass kernel, per tile (global timer, ns): [0] tile + 1; coordinator:
// [1] tile folded, [2] incoming state resolved, [3] group states posted; first compute warp:
// [4] iteration start, [5] next ticket known, [6] particular pass done, [7] lane scan done, [8] fold
// done; correction of the tile: [9] start, [10] group state observed, [11] row states stored,
// [12] stored; [13] SM id; [14] stash start, [15] input stashed.
// Phase trace of the tensor-core kernel, per tile (global timer, ns): [0] tile + 1, [13] SM id;
// coordinator: [1] tile folded, [2] incoming state resolved, [3] group states posted; producer:
// [16] ticket drawn, [17] unit 0 loads issued; MMA issuer: [18] unit 0 first products issued,
// [19] unit 0 remainder products issued, [20] unit 0 correction issued; [21] unit 0 remainder formed;
// epilogue warp of group 0: [4] accumulator observed, [7] lane scan done, [8] fold done, [9]
// correction start, [10] group state observed, [11] state operand posted, [12] correction observed,
// [14] outputs stored; epilogue warp of group 4: [22] accumulator observed, [23] lane scan done,
// [24] correction observed, [25] outputs stored.
template <int K, int N, int W>
cudaError_t launch_lane(bool norm, const LaneParams<K> &p, long long grid, cudaStream_t s);
#define SOSK_DECLARE_LANE(K, N, W) \
    template <>                    \
    cudaError_t launch_lane<K, N, W>(bool norm, const LaneParams<K> &p, long long grid, cudaStream_t s);
#define SOSK_DECLARE_LANE_NW(N, W)                                                                          \
    SOSK_DECLARE_LANE(1, N, W) SOSK_DECLARE_LANE(2, N, W) SOSK_DECLARE_LANE(3, N, W) SOSK_DECLARE_LANE(4, N, W) \
    SOSK_DECLARE_LANE(5, N, W) SOSK_DECLARE_LANE(6, N, W) SOSK_DECLARE_LANE(7, N, W) SOSK_DECLARE_LANE(8, N, W)
SOSK_DECLARE_LANE_NW(32, 7)
SOSK_DECLARE_LANE_NW(64, 7)
SOSK_DECLARE_LANE_NW(64, 10)
// Thread blocks of the skewed-pass kernel (N samples per lane, W groups per tile) that fit on one SM
// (0 if unavailable).
int lane_blocks_per_sm(int K, int N, int W, bool norm);

// ---- PH kernel on the tensor cores (sosfilt_tc.cuh): N = 64 samples per lane, tiles of kTcGroups
// groups; x and y 16-byte aligned and n >= 64.  img: the constant operands' shared-memory image
// (tc_image_bytes), gtail: [2K][64] state responses in float32.
constexpr int kTcGroups = 8;
constexpr int kTcImageBytes = 49152;
template <int K>
cudaError_t launch_tc(const LaneParams<K> &p, const float *img, const float *gtail, long long grid, cudaStream_t s);
#define SOSK_DECLARE_TC(K) \
    template <>            \
    cudaError_t launch_tc<K>(const LaneParams<K> &p, const float *img, const float *gtail, long long grid, cudaStream_t s);
SOSK_DECLARE_TC(1) SOSK_DECLARE_TC(2) SOSK_DECLARE_TC(3) SOSK_DECLARE_TC(4)
SOSK_DECLARE_TC(5) SOSK_DECLARE_TC(6) SOSK_DECLARE_TC(7) SOSK_DECLARE_TC(8)
#undef SOSK_DECLARE_TC
int tc_blocks_per_sm(int K);

// ---- multi-signal persistent kernel (sosfilt_batch.cuh): the PH kernel with a skewed particular
// pass over a global queue of (signal, tile) work items.  Two tile geometries, chosen per signal:
// N = 64 or N = 32 samples per lane, kBatchW groups (compute warps) per tile either way, so that
// both run in blocks of the same shape and one launch serves every class.
constexpr int kBatchN = 64;      // samples per lane of the wide geometry
constexpr int kBatchNs = 32;     // samples per lane of the short geometry (tiles of half the samples)
constexpr int kBatchW = kLaneW;  // groups (compute warps) per tile: the tables of the PH kernel
constexpr int kBatchGeoms = 2;   // geometry 0: N = kBatchN, geometry 1: N = kBatchNs
#if defined(__CUDACC__)
#define SOSK_HD __host__ __device__
#else
#define SOSK_HD
#endif
SOSK_HD constexpr int batch_geom_n(int geom) { return geom == 0 ? kBatchN : kBatchNs; }

// One signal of a batch (device array, built by the host for each batched run).
struct BatchSig {
    const float *x;
    float *y;
    long long n, G;        // samples, groups of 32 N samples (N of the signal's class)
    long long tile0;       // first global tile of the signal; its tiles are tile0 .. tile0 + ceil(G / W) - 1
    const float *zi;       // device [K][2] initial state (true domain) or nullptr
    float *zf;             // device [K][2] final state or nullptr
    const LaneSec *sec;    // device [K] section constants for the class's N
    const float4 *MX;      // device coupling blocks of M_N (as LaneParams::MX)
    const float *tab;      // device table block (LaneDims<K, N>::TAB_GLOBAL floats)
    const float *Mm;       // device [kBatchN][2K(K+1)] packed one-sample transition powers M1^(m+1)
    float gain;            // input multiplier (product of the b0 when normalized)
    int aligned;           // x and y 16-byte aligned
};

template <int K>
struct BatchParams {
    const BatchSig *sigs;
    const int *tile_sig;        // [n_tiles] signal of each global tile
    long long n_tiles;
    unsigned long long *desc;   // [n_tiles][2][2K] tagged carry words: local, resolved
    unsigned long long *ticket;
    unsigned long long ticket_base;
    unsigned int epoch;
    int *status;
    long long spin_budget;
};

// One class's queue in the single-kernel batch (the fields of BatchParams that do not depend on K).
struct BatchQueue {
    const BatchSig *sigs;
    const int *tile_sig;
    long long n_tiles;
    unsigned long long *desc;
    unsigned long long *ticket;
    unsigned long long ticket_base;
    unsigned int epoch;
};

// Class of a batched signal: geometry, section count K = 1..8 and b0 handling,
// code = 16 geometry + 2 (K - 1) + b0-normalized.
constexpr int kBatchClassesMax = 16 * kBatchGeoms;
SOSK_HD constexpr int batch_class(int geom, int K, bool norm) { return 16 * geom + 2 * (K - 1) + (norm ? 1 : 0); }
SOSK_HD constexpr int batch_class_k(int code) { return ((code & 15) >> 1) + 1; }
SOSK_HD constexpr int batch_class_geom(int code) { return code >> 4; }

struct BatchAllParams {
    int n_classes;
    int code[kBatchClassesMax];         // class code (batch_class)
    int blk_off[kBatchClassesMax + 1];  // blocks [blk_off[c], blk_off[c + 1]) start on class c
    BatchQueue q[kBatchClassesMax];
    int *status;
    long long spin_budget;
};

// Launch the single persistent kernel over every class of a batch (sosfilt_batch_all.cu).
cudaError_t launch_batch_all(const BatchAllParams &p, long long grid, cudaStream_t s);
int batch_all_blocks_per_sm();

// Device memory for the lookback descriptors and the ticket counter of one cascade run.
struct Scratch {
    unsigned long long *desc;
    size_t desc_words;
    unsigned long long *ticket;
};

// Launch one pass.  Returns cudaSuccess or the launch error.
// lbm: predecessors read per lookback round / 32 (0 = the default for N).
cudaError_t launch_dccr(int K, int N, bool norm, int lbm, const PassParams &p, long long grid, cudaStream_t s);
int default_lbm(int N);

}  // namespace sosk
