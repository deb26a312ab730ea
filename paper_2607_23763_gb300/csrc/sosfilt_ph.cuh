// Persistent single-signal kernel: PH factorization of every lane's block (Sec. II-C) with one
// carry per tile for the whole cascade, sm_103a.
//
// A tile is W = kPhWc consecutive groups of C = 32 N samples (N = kPhN); compute warp w of a thread
// block filters group w of the tile, lane l the samples l N .. l N + N - 1.  Per tile:
//   1. particular solution: every lane runs its N samples through the whole cascade from zero state
//      (the forward substitution of Sec. II-C with zero initial blocks), as a wavefront: four or eight
//      samples at a time pass through all K sections, whose direct-form histories (x[-1], x[-2],
//      w[-1], w[-2]) stay in registers; the samples themselves stay in the lane's row of shared
//      memory and are overwritten in place by the particular output.
//   2. lane scan (Sec. II-C's recursive doubling, Kogge-Stone over the 32 lanes) on the whole
//      cascade state: lane l's incoming state S_l obeys S_{l+1} = M_N S_l + t_l, t_l the lane's
//      terminal particular state and M_N the cascade's zero-input transition over N samples.  M_N
//      is block lower-triangular, so section k's words are scanned with its own (T^N)^(2^r) once
//      the lower sections' words are known and their coupling blocks are folded into t_l.  The
//      by-product is the group's local carry (its state after the last sample under zero incoming
//      group state).
//   3. a coordinator warp folds the tile's local carries, publishes the tile carry and resolves the
//      tile's incoming 2K-word state by decoupled lookback over tiles (Sec. IV-B, Eq. 25 on the
//      cascade state), then derives every group's incoming state Z.
//   4. homogeneous correction, once for the whole cascade: lane l's true incoming state is
//      S_l + (M_N)^l Z and its output at sample m gains sum_j H_j(m) [S_l + (M_N)^l Z]_j, H_j the
//      cascade's zero-input output from unit state j (Eq. 24 in cascade form).  Lane-level and
//      group-level corrections are one pass over the samples.
// The particular output of tile t leaves for y at once and the lanes' scan states go to a small
// per-block ring in global memory; tile t is corrected after the pass of tile t + kPhR - 1, reading
// its particular output back from L2, so the coordinator has that many tiles' time to resolve it and
// the compute warps do not wait on the lookback.  Tiles come from an ascending ticket counter
// (Sec. IV-A); the first warp of a block to start tile t draws the ticket of tile t + 2.  Inputs are
// prefetched one tile ahead with cp.async into the other of the warp's two row buffers; stores
// are coalesced 128-bit writes of rows transposed through shared memory.  Arithmetic is scalar
// FP32 FMA: on this GPU the packed f32x2 form has the same FMA rate and takes the issue slot for
// two cycles.
#pragma once
#include "sosfilt_cascade.cuh"

namespace sosk {

template <int K>
struct PhDims {
    static constexpr int S = 2 * K;
    static constexpr int NB = K * (K + 1) / 2;
    static constexpr int NF = 4 * NB;  // floats of one packed lower block-triangular matrix
    // per-lane stride of (M_N)^lane and (A_T)^lane: an odd number of 16-byte words, so that the
    // lanes' 128-bit reads of their own rows fall in distinct banks
    static constexpr int MS = ((NF / 4) & 1) ? NF : NF + 4;
    static constexpr int FULL = S * S;
    static constexpr int P2 = S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;
    static constexpr int SH = 5 - (P2 == 2 ? 1 : P2 == 4 ? 2 : P2 == 8 ? 3 : 4);
    // global table block: (M_N)^lane [32][MS], (A_T)^lane [32][MS] (packed), A_C dense
    // column-major, then A_T dense and (A_T)^(32 w), w = 1..kMaxWin, dense
    static constexpr int OFF_ATL = 32 * MS;
    static constexpr int OFF_AC = OFF_ATL + 32 * MS;
    static constexpr int OFF_AT = OFF_AC + FULL;
    static constexpr int TAB_GLOBAL = OFF_AT + (1 + kMaxWin) * FULL;
};

// Direct-form history of one section over the lane's samples: inputs x[-1], x[-2] and outputs
// w[-1], w[-2], zero at the lane's first sample.
struct PhHist {
    float x1, x2, w1, w2;
};

// One sample through section k: w = b0 x + b1 x[-1] + b2 x[-2] - a1 w[-1] - a2 w[-2].  The terms of
// older samples are summed first, so only two operations follow the arrival of x and one the
// arrival of w[-1] (the wavefront's critical path).
template <int K, bool NORM>
__device__ __forceinline__ float ph_step(const PhParams<K> &p, int k, PhHist &h, float x) {
    const float4 c0 = p.sec[k].c0;  // b0, b1, b2, -a1 (compile-time k: constant-bank operands)
    const float na2 = p.sec[k].c1.x;
    const float old = fmaf(c0.y, h.x1, fmaf(c0.z, h.x2, na2 * h.w2));
    const float v = NORM ? x + old : fmaf(c0.x, x, old);
    const float w = fmaf(c0.w, h.w1, v);
    h.x2 = h.x1;
    h.x1 = x;
    h.w2 = h.w1;
    h.w1 = w;
    return w;
}

// Transposed direct form II state of section k after the latest sample of its history.
template <int K>
__device__ __forceinline__ void ph_state(const PhParams<K> &p, int k, const PhHist &h, float &z1, float &z2) {
    const float4 c0 = p.sec[k].c0;
    const float na2 = p.sec[k].c1.x;
    z1 = fmaf(c0.y, h.x1, fmaf(c0.z, h.x2, fmaf(c0.w, h.w1, na2 * h.w2)));
    z2 = fmaf(c0.z, h.x1, na2 * h.w1);
}

// Particular solution of the lane's row (N samples, in place) through all K sections from zero
// state; t receives the terminal state, and with CAPTURE the lane `cap_lane` writes its state after
// sample m_last to cap (shared memory).
template <int K, int N, bool NORM, bool CAPTURE>
__device__ __forceinline__ void ph_particular(const PhParams<K> &p, float *row, float gain, float (&t)[2 * K],
                                              int m_last, bool cap_lane, float *cap) {
    constexpr int U = K <= 4 ? 4 : 8;  // samples per step of the wavefront
    PhHist h[K];
#pragma unroll
    for (int k = 0; k < K; ++k) h[k] = PhHist{0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int q = 0; q < N; q += U) {
        float v[U];
#pragma unroll
        for (int i = 0; i < U; i += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(row + q + i);
            v[i] = a.x;
            v[i + 1] = a.y;
            v[i + 2] = a.z;
            v[i + 3] = a.w;
        }
#pragma unroll
        for (int i = 0; i < U; ++i) {
            if (NORM) v[i] *= gain;
#pragma unroll
            for (int k = 0; k < K; ++k) v[i] = ph_step<K, NORM>(p, k, h[k], v[i]);
            if constexpr (CAPTURE) {
                if (q + i == m_last && cap_lane) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float z1, z2;
                        ph_state<K>(p, k, h[k], z1, z2);
                        cap[2 * k] = z1;
                        cap[2 * k + 1] = z2;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < U; i += 4)
            *reinterpret_cast<float4 *>(row + q + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) ph_state<K>(p, k, h[k], t[2 * k], t[2 * k + 1]);
}

// Cascade lane scan: from the lanes' terminal particular states t, the lane's incoming state S
// (exclusive, relative to zero group state) and, in lane 31, the group's local carry a_out.
template <int K>
__device__ __forceinline__ void ph_scan(const PhParams<K> &p, const float (&t)[2 * K], float (&S)[2 * K],
                                        float *a_out, int lane) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float u1 = t[2 * k], u2 = t[2 * k + 1];
        // couple the lane states of sections j < k: u += M_N[k][j] S_l[j]
#pragma unroll
        for (int j = 0; j < k; ++j) {
            const float4 b = p.MX[k * (k - 1) / 2 + j];
            u1 = fmaf(b.x, S[2 * j], fmaf(b.y, S[2 * j + 1], u1));
            u2 = fmaf(b.z, S[2 * j], fmaf(b.w, S[2 * j + 1], u2));
        }
        // inclusive scan over the lanes: E_l = T^N E_{l-1} + u_l
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const float o1 = __shfl_up_sync(0xffffffffu, u1, 1 << r);
            const float o2 = __shfl_up_sync(0xffffffffu, u2, 1 << r);
            const float4 tn = p.sec[k].tn[r];
            if (lane >= (1 << r)) {
                u1 = fmaf(tn.x, o1, fmaf(tn.y, o2, u1));
                u2 = fmaf(tn.z, o1, fmaf(tn.w, o2, u2));
            }
        }
        float s1 = __shfl_up_sync(0xffffffffu, u1, 1), s2 = __shfl_up_sync(0xffffffffu, u2, 1);
        if (lane == 0) s1 = s2 = 0.f;
        S[2 * k] = s1;
        S[2 * k + 1] = s2;
        if (lane == 31) {
            a_out[2 * k] = u1;
            a_out[2 * k + 1] = u2;
        }
    }
}

// y += A x for a packed lower block-triangular A and x both in shared memory (x read as word
// pairs, broadcast).
template <int K>
__device__ __forceinline__ void packed_mv_acc_ss(const float *__restrict__ A, const float *__restrict__ x,
                                                 float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = y[2 * s], y1 = y[2 * s + 1];
#pragma unroll
        for (int t = 0; t <= s; ++t) {
            const float4 B = *reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + t));
            const float2 xt = *reinterpret_cast<const float2 *>(x + 2 * t);
            y0 = fmaf(B.x, xt.x, fmaf(B.y, xt.y, y0));
            y1 = fmaf(B.z, xt.x, fmaf(B.w, xt.y, y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
    }
}

// y = A x for a packed lower block-triangular A in global memory, one section at a time.
template <int K>
__device__ __forceinline__ void packed_mv_g(const float *__restrict__ A, const float (&x)[2 * K], float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int t = 0; t <= s; ++t) {
            const float4 B = __ldg(reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + t)));
            y0 = fmaf(B.x, x[2 * t], fmaf(B.y, x[2 * t + 1], y0));
            y1 = fmaf(B.z, x[2 * t], fmaf(B.w, x[2 * t + 1], y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
        asm volatile("" ::: "memory");
    }
}

template <int K, bool NORM>
__global__ void __maxnreg__(K <= 4 ? 80 : 128) sos_ph_kernel(const __grid_constant__ PhParams<K> p) {
    using Dm = PhDims<K>;
    constexpr int S = Dm::S, N = kPhN, W = kPhWc, R = kPhR;
    constexpr int P = N + 4;  // padded row pitch (floats): conflict-free 128-bit row access
    constexpr int C = N * kL;
    // (A_T)^lane in shared memory too when two blocks share an SM (K >= 5)
    constexpr bool kAtlShared = K >= 5;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);  // [W][2][32][P]: two row buffers per warp
    float *sMl = rows + W * 2 * kL * P;              // (M_N)^lane [32][MS] (packed)
    float *sATl = sMl + 32 * Dm::MS;                 // (A_T)^lane [32][MS] when kAtlShared
    float *sACd = sATl + (kAtlShared ? 32 * Dm::MS : 0);  // A_C dense column-major
    float *a_buf = sACd + Dm::FULL;                  // [R][W][S] local carries
    float *z_buf = a_buf + R * W * S;                // [R][W][S] incoming states
    float *zs_tail = z_buf + R * W * S;              // [S] lane-local final state
    float *agg = zs_tail + S;                        // [R][S] tile carry, zero state
    // tiles in flight use slot it % R; tickets a ring of 8 (drawn two tiles ahead)
    __shared__ unsigned long long bar_local[R], bar_zready[R], bar_ticket[8];
    __shared__ long long ring[8];
    __shared__ int fold_count[R];
    __shared__ unsigned draw_count[8];
    __shared__ int tickets_exhausted;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long budget = p.spin_budget;
    const float *gATl = p.tab + Dm::OFF_ATL;
    const float *gATd = p.tab + Dm::OFF_AT;

    for (int i = threadIdx.x; i < Dm::FULL; i += blockDim.x) sACd[i] = __ldg(p.tab + Dm::OFF_AC + i);
    for (int i = threadIdx.x; i < 8 * Dm::MS; i += blockDim.x)
        reinterpret_cast<float4 *>(sMl)[i] = __ldg(reinterpret_cast<const float4 *>(p.tab) + i);
    if constexpr (kAtlShared) {
        for (int i = threadIdx.x; i < 8 * Dm::MS; i += blockDim.x)
            reinterpret_cast<float4 *>(sATl)[i] = __ldg(reinterpret_cast<const float4 *>(gATl) + i);
    }
    auto draw_ticket = [&]() -> long long {
        if (tickets_exhausted) return -1;
        long long t = static_cast<long long>(atomicAdd(p.ticket, 1ULL) - p.ticket_base);
        if (t >= p.n_tiles) {
            tickets_exhausted = 1;
            t = -1;
        }
        return t;
    };
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            mbar_init(&bar_local[i], 1);
            mbar_init(&bar_zready[i], 1);
            fold_count[i] = 0;
        }
        tickets_exhausted = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            mbar_init(&bar_ticket[i], 1);
            draw_count[i] = 0;
        }
        ring[0] = draw_ticket();
        ring[1] = draw_ticket();
        mbar_arrive(&bar_ticket[0]);
        mbar_arrive(&bar_ticket[1]);
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------------ coordinator warp
        const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
        auto zinit = [&](int i) -> float { return p.zi ? p.zi[i] * p.sec[i >> 1].c1.y : 0.f; };
        unsigned it = 0;
        for (;;) {
            const unsigned slot = it % R, ph = (it / R) & 1;
            if (!mbar_wait_backoff(&bar_ticket[it & 7], (it >> 3) & 1, budget, p.status, 1024)) break;
            const long long cur = ring[it & 7];
            if (cur < 0) break;
            if (!mbar_wait_backoff(&bar_local[slot], ph, budget, p.status, 1024)) break;
            unsigned long long *tr = (p.trace && lane == 0 && cur < p.trace_tiles)
                                         ? p.trace + static_cast<size_t>(cur) * kTraceSlots
                                         : nullptr;
            if (tr) {
                unsigned smid;
                asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
                tr[0] = static_cast<unsigned long long>(cur) + 1;
                tr[1] = global_ns();
                tr[11] = smid;
                tr[12] = blockIdx.x;
            }
            const float *abuf = a_buf + slot * W * S;
            const float acc_i = agg[slot * S + (lane < S ? lane : 0)];
            float tmp[S];
            if (tr) tr[2] = global_ns();
            unsigned long long *dcur = p.desc + static_cast<size_t>(cur) * S;
            float zi_lane = 0.f;
            unsigned n_win = 0, n_wait = 0;
            if (cur == 0) {
                zi_lane = zinit(lane < S ? lane : 0);
            } else {
                // decoupled lookback over tiles, 32 predecessors per round
                const long long t_start = clock64();
                int win = 0;
                unsigned nap = 64;
                for (;;) {
                    const long long pred = cur - 1 - 32LL * win - lane;
                    float v[S];
                    int st;
                    if (pred >= 0) {
                        const unsigned long long *dp = p.desc + static_cast<size_t>(pred) * S;
                        bool allG = true, allL = true;
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const unsigned long long wd = ld_relaxed_b64(dp + i);
                            const unsigned tg = static_cast<unsigned>(wd >> 32);
                            allG = allG && (tg == tagG);
                            allL = allL && (tg == tagL);
                            v[i] = __uint_as_float(static_cast<unsigned>(wd));
                        }
                        st = allG ? 2 : (allL ? 1 : 0);
                    } else {
                        st = 2;
#pragma unroll
                        for (int i = 0; i < S; ++i) v[i] = (pred == -1) ? zinit(i) : 0.f;
                    }
                    const unsigned glob = __ballot_sync(0xffffffffu, st == 2);
                    const unsigned inv = __ballot_sync(0xffffffffu, st == 0);
                    const int j = glob ? __ffs(glob) - 1 : 32;
                    const unsigned need = (j >= 31) ? 0xffffffffu : ((2u << j) - 1u);
                    if (inv & need) {
                        ++n_wait;
                        if (__any_sync(0xffffffffu, (clock64() - t_start) > budget)) {
                            if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                            break;
                        }
                        __nanosleep(nap);  // back off: the result is needed two tiles later
                        nap = nap < 2048 ? 2 * nap : 2048;
                        continue;
                    }
                    ++n_win;
                    if (lane > j) {
#pragma unroll
                        for (int i = 0; i < S; ++i) v[i] = 0.f;
                    }
                    if constexpr (kAtlShared)
                        packed_mv<K>(sATl + lane * Dm::MS, v, tmp);
                    else
                        packed_mv_g<K>(gATl + lane * Dm::MS, v, tmp);
                    float part = reduce_scatter<S, Dm::P2, Dm::SH>(tmp, lane);
                    part = __shfl_sync(0xffffffffu, part, (lane < S ? lane : 0) << Dm::SH);
                    if (win == 0) {
                        zi_lane += part;
                    } else {
                        const float *Aw = gATd + win * Dm::FULL;
                        float y = 0.f;
                        const int row = lane < S ? lane : 0;
#pragma unroll
                        for (int jj = 0; jj < S; ++jj)
                            y = fmaf(__ldg(Aw + jj * S + row), __shfl_sync(0xffffffffu, part, jj), y);
                        zi_lane += y;
                    }
                    if (j < 32) break;
                    if (++win > kMaxWin) {
                        if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                        break;
                    }
                }
            }
            if (tr) {
                tr[3] = global_ns();
                tr[5] = (static_cast<unsigned long long>(n_wait) << 32) | n_win;
            }
            if (cur + 1 < p.n_tiles) {
                float gl = acc_i;
                const int row = lane < S ? lane : 0;
#pragma unroll
                for (int jj = 0; jj < S; ++jj)
                    gl = fmaf(__ldg(gATd + jj * S + row), __shfl_sync(0xffffffffu, zi_lane, jj), gl);
                if (lane < S) st_relaxed_b64(dcur + lane, pack_word(tagG, gl));
            }
            // incoming state of each group: Z_0 = Z, Z_{v+1} = A_C Z_v + a_v
            float *zb = z_buf + slot * W * S;
#pragma unroll 1
            for (int v = 0; v < W; ++v) {
                if (lane < S) zb[v * S + lane] = zi_lane;
                if (v + 1 < W) zi_lane = lane_mv<S>(sACd, zi_lane, lane) + abuf[v * S + (lane < S ? lane : 0)];
            }
            __syncwarp();
            // one barrier per slot: the pass of tile it + R waits for the correction of tile it, so a
            // slot's barrier never runs two phases ahead of a waiter
            if (lane == 0) mbar_arrive(&bar_zready[slot]);
            if (tr) tr[4] = global_ns();
            ++it;
        }
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int w = warp - 1;
    float *B0 = rows + w * 2 * kL * P;  // the warp's two row buffers (B0, B0 + 32 P)
    float2 *gring = p.sring + (static_cast<size_t>(blockIdx.x) * R * W + w) * K * 32;  // slot stride W K 32
    const bool want_zf = p.zf != nullptr;
    const long long g_last = p.G - 1;
    const long long p_last = p.n - 1 - g_last * C;
    const int lane_last = static_cast<int>(p_last / N);
    const int m_last = p.m_last;

    auto issue_load = [&](long long tile, float *X) {
        const long long base = (tile * W + w) * C;
        const long long avail = p.n - base;
        if (avail >= C && p.aligned) {
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const int off = 4 * (j * 32 + lane);
                cp_async16(X + (off / N) * P + (off % N), p.x + base + off);
            }
            cp_async_commit();
        } else {
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const int off = 4 * (j * 32 + lane);
                const float *src = p.x + base + off;
                float4 v;
                v.x = (off + 0 < avail) ? __ldcs(src + 0) : 0.f;
                v.y = (off + 1 < avail) ? __ldcs(src + 1) : 0.f;
                v.z = (off + 2 < avail) ? __ldcs(src + 2) : 0.f;
                v.w = (off + 3 < avail) ? __ldcs(src + 3) : 0.f;
                *reinterpret_cast<float4 *>(X + (off / N) * P + (off % N)) = v;
            }
        }
    };

    // The rows of buffer Y (lane l: samples l N .. l N + N - 1 of group g) to y, read back transposed
    // so that each 128-bit store instruction of the warp covers 512 contiguous bytes; bounded for a
    // partial group.
    auto store_rows = [&](long long g, const float *Y, bool streaming) {
        __syncwarp();
        if (g < p.G) {
            const long long base = g * C;
            const long long avail = p.n - base;
            if (avail >= C && p.aligned) {
#pragma unroll
                for (int j = 0; j < N / 4; ++j) {
                    const int off = 4 * (j * 32 + lane);
                    const float4 v = *reinterpret_cast<const float4 *>(Y + (off / N) * P + (off % N));
                    float4 *dst = reinterpret_cast<float4 *>(p.y + base + off);
                    if (streaming)
                        __stcs(dst, v);
                    else
                        *dst = v;
                }
            } else {
#pragma unroll
                for (int j = 0; j < N / 4; ++j) {
                    const int off = 4 * (j * 32 + lane);
                    const float4 v = *reinterpret_cast<const float4 *>(Y + (off / N) * P + (off % N));
                    float *dst = p.y + base + off;
                    if (off + 0 < avail) dst[0] = v.x;
                    if (off + 1 < avail) dst[1] = v.y;
                    if (off + 2 < avail) dst[2] = v.z;
                    if (off + 3 < avail) dst[3] = v.w;
                }
            }
        }
        __syncwarp();
    };

    auto wtrace = [&](long long tile, int slot) {
        if (p.trace && w == 0 && lane == 0 && tile < p.trace_tiles)
            p.trace[static_cast<size_t>(tile) * kTraceSlots + slot] = global_ns();
    };

    // Correction of the tile of iteration jt (kPhR - 1 iterations back), in buffer Y: its particular
    // output is read back from y (L2), the lane's true incoming state is S_l + (M_N)^lane Z, and the
    // corrected rows leave for y.
    auto correct_and_store = [&](long long tile, unsigned jt, float *Y) -> bool {
        const unsigned slot = jt % R;
        wtrace(tile, 8);
        if (!mbar_wait_backoff(&bar_zready[slot], (jt / R) & 1, budget, p.status, 512)) return false;
        wtrace(tile, 9);
        const long long g = tile * W + w;
        const float2 *gS = gring + static_cast<size_t>(slot) * W * K * 32;
        float dz[S];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 q = __ldcg(gS + k * 32 + lane);
            dz[2 * k] = q.x;
            dz[2 * k + 1] = q.y;
        }
        packed_mv_acc_ss<K>(sMl + lane * Dm::MS, z_buf + (slot * W + w) * S, dz);
        if (want_zf && g == g_last && lane == lane_last) {
            // final state: lane-local state after the last sample plus the transition of the lane's
            // incoming state over the samples up to it
            float zt[S];
            packed_mv_param<K>(p.A_tail, dz, zt);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const float inv = p.sec[s].c1.z;
                p.zf[2 * s] = (zs_tail[2 * s] + zt[2 * s]) * inv;
                p.zf[2 * s + 1] = (zs_tail[2 * s + 1] + zt[2 * s + 1]) * inv;
            }
        }
        if (g < p.G) {
            const long long base = g * C;
            const long long avail = p.n - base;
            // the particular output of this group, written by this warp kPhR - 1 iterations ago: read back
            // from L2 with coalesced loads, transposed into rows
            wtrace(tile, 19);
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const int off = 4 * (j * 32 + lane);
                const float *src = p.y + base + off;
                float4 v;
                if (avail >= C && p.aligned) {
                    v = __ldcg(reinterpret_cast<const float4 *>(src));
                } else {
                    v.x = (off + 0 < avail) ? __ldcg(src + 0) : 0.f;
                    v.y = (off + 1 < avail) ? __ldcg(src + 1) : 0.f;
                    v.z = (off + 2 < avail) ? __ldcg(src + 2) : 0.f;
                    v.w = (off + 3 < avail) ? __ldcg(src + 3) : 0.f;
                }
                *reinterpret_cast<float4 *>(Y + (off / N) * P + (off % N)) = v;
            }
            __syncwarp();
            float *row = Y + lane * P;
#pragma unroll
            for (int q = 0; q < N / 4; ++q) {
                float4 v = *reinterpret_cast<const float4 *>(row + 4 * q);
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    v.x = fmaf(p.H[j][4 * q + 0], dz[j], v.x);
                    v.y = fmaf(p.H[j][4 * q + 1], dz[j], v.y);
                    v.z = fmaf(p.H[j][4 * q + 2], dz[j], v.z);
                    v.w = fmaf(p.H[j][4 * q + 3], dz[j], v.w);
                }
                *reinterpret_cast<float4 *>(row + 4 * q) = v;
            }
            wtrace(tile, 20);
        }
        store_rows(g, Y, true);
        wtrace(tile, 10);
        return true;
    };

    if (!mbar_wait_backoff(&bar_ticket[0], 0, budget, p.status, 256)) return;
    long long tile = ring[0];
    if (tile < 0) return;
    issue_load(tile, B0);
    unsigned it = 0;
    constexpr int LAG = R - 1;  // tile of iteration it is corrected in iteration it + LAG
    long long pend[R];          // tile of iteration i at pend[i % R], awaiting correction
    bool ok = true;
    for (;;) {
        const long long g = tile * W + w;
        const unsigned slot = it % R;
        float *X = B0 + (it & 1) * kL * P;        // this tile's rows (prefetched)
        float *Xn = B0 + ((it & 1) ^ 1) * kL * P;  // the other buffer: next tile's prefetch
        wtrace(tile, 13);
        cp_async_wait_all();
        __syncwarp();
        wtrace(tile, 14);
        if (!mbar_wait_backoff(&bar_ticket[(it + 1) & 7], ((it + 1) >> 3) & 1, budget, p.status, 256)) {
            ok = false;
            break;
        }
        const long long next = ring[(it + 1) & 7];
        wtrace(tile, 15);
        if (next >= 0) issue_load(next, Xn);
        // the first warp to start this iteration draws the ticket of iteration it + 2 (its result is
        // used after the pass, which hides the atomic's latency)
        bool drawer = false;
        long long drawn = -1;
        if (next >= 0) {
            unsigned c = 0;
            if (lane == 0) c = atomicAdd(&draw_count[(it + 2) & 7], 1u);
            drawer = (__shfl_sync(0xffffffffu, c, 0) % W) == 0;
            if (drawer && lane == 0) drawn = draw_ticket();
        }

        wtrace(tile, 6);
        {
            float t[S], Sl[S];
            if (want_zf && g == g_last)
                ph_particular<K, N, NORM, true>(p, X + lane * P, p.gain, t, m_last, lane == lane_last, zs_tail);
            else
                ph_particular<K, N, NORM, false>(p, X + lane * P, p.gain, t, m_last, false, nullptr);
            ph_scan<K>(p, t, Sl, a_buf + (slot * W + w) * S, lane);
            float2 *gS = gring + static_cast<size_t>(slot) * W * K * 32;
#pragma unroll
            for (int k = 0; k < K; ++k) gS[k * 32 + lane] = make_float2(Sl[2 * k], Sl[2 * k + 1]);
        }
        wtrace(tile, 7);
        {
            // the last warp of the tile to finish folds the groups' local carries (c = a_0;
            // c = A_C c + a_v) and posts the tile's carry
            __syncwarp();
            int old = 0;
            if (lane == 0) {
                __threadfence_block();
                old = atomicAdd(&fold_count[slot], 1);
            }
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == W - 1) {
                __threadfence_block();
                const float *abt = a_buf + slot * W * S;
                const int li = lane < S ? lane : 0;
                float c = abt[li];
#pragma unroll 1
                for (int v = 1; v < W; ++v) c = lane_mv<S>(sACd, c, lane) + abt[v * S + li];
                if (tile > 0 && lane < S)
                    st_relaxed_b64(p.desc + static_cast<size_t>(tile) * S + lane, pack_word((p.epoch << 2) | 1u, c));
                if (lane < S) agg[slot * S + lane] = c;
                if (lane == 0) fold_count[slot] = 0;
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_local[slot]);
            }
        }
        if (next < 0) {
            // no further tiles: post the end marker for iteration it + 2 (once per block)
            if (lane == 0 && atomicAdd(&draw_count[(it + 2) & 7], 1u) % W == 0) {
                ring[(it + 2) & 7] = -1;
                mbar_arrive(&bar_ticket[(it + 2) & 7]);
            }
        } else if (drawer && lane == 0) {
            ring[(it + 2) & 7] = drawn;
            mbar_arrive(&bar_ticket[(it + 2) & 7]);
        }
        // the particular output leaves at once; the buffer is then reused for the correction
        wtrace(tile, 16);
        store_rows(g, X, false);
        wtrace(tile, 18);
        pend[it % R] = tile;
        if (it >= static_cast<unsigned>(LAG) && !correct_and_store(pend[(it - LAG) % R], it - LAG, X)) {
            ok = false;
            break;
        }
        if (next < 0) break;
        tile = next;
        ++it;
    }
    // the last tiles, in order; the buffer of the last iteration is free
    float *Xf = B0 + (it & 1) * kL * P;
    const unsigned first = it >= static_cast<unsigned>(LAG) ? it - LAG + 1 : 0;
    for (unsigned j = first; ok && j <= it; ++j) ok = correct_and_store(pend[j % R], j, Xf);
}

template <int K>
constexpr size_t ph_smem_bytes() {
    using Dm = PhDims<K>;
    constexpr int W = kPhWc, R = kPhR;
    return sizeof(float) * (static_cast<size_t>(W) * 2 * kL * (kPhN + 4)) +
           sizeof(float) * (32 * Dm::MS * (K >= 5 ? 2 : 1)) +
           sizeof(float) * (Dm::FULL + R * W * Dm::S + R * W * Dm::S + Dm::S + R * Dm::S);
}

}  // namespace sosk
