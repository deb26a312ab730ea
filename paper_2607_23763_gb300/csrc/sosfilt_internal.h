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

// Device status bits (sticky, OR-ed by the kernels).
constexpr int kDevErrTimeout = 1;

// Per-section tables, float32, derived in float64 on the host for one N.
// Level i of the reduction holds y[m] + e_i y[m - 2^i] + f_i y[m - 2^(i+1)] = v_i[m].
struct SecCoef {
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

// Launch one pass.  Returns cudaSuccess or the launch error.
// lbm: predecessors read per lookback round / 32 (0 = the default for N).
cudaError_t launch_dccr(int K, int N, bool norm, int lbm, const PassParams &p, long long grid, cudaStream_t s);
int default_lbm(int N);

}  // namespace sosk
