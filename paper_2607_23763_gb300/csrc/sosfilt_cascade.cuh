// Persistent single-signal kernel with one carry per tile for the whole cascade, sm_103a.
//
// A tile is W consecutive groups of C = 32*N samples (Sec. IV-A); warp w of a thread block
// owns group w of the tile, lane l the samples l*N .. l*N+N-1 of the group.  Per tile:
//   1. zero-state pass: each compute warp filters its group through all K sections in
//      registers with zero incoming group state (divide-and-conquer cyclic reduction per
//      section, Sec. II-E; the lanes' states are scanned inside the warp with T^N).  The pass
//      touches no global memory and no block barrier.  Its by-product is the group's local
//      carry: the 2K-word cascade state at the group's end under zero incoming state.
//   2. one coordinator warp per block folds the W local carries into the tile's carry with the
//      group transition A_C, publishes it, resolves the tile's incoming 2K-word state by
//      decoupled lookback over tiles with the tile transition A_T = A_C^W (Sec. II-F, Eq. 25
//      with the cascade state in place of one section's; Sec. IV-B), publishes the resolved
//      carry and derives each group's incoming state.
//   3. correction: by linearity the true output is the zero-state output plus the zero-input
//      response of the cascade from the group's incoming state Z (the homogeneous correction of
//      Eq. 24, once for the whole cascade): lane l's state is (M_N)^l Z and the output at its
//      sample m gains sum_j H_j(m) [(M_N)^l Z]_j.
// The coordinator resolves tile t while the compute warps already run tile t+1: the lookback's
// memory latency is off the critical path.  Tiles are drawn from an ascending ticket counter,
// so every tile's predecessors are held by running or finished blocks (Sec. IV-A).
// Inputs are prefetched one tile ahead with cp.async; outputs leave by bulk (TMA) stores.
#pragma once
#include "sosfilt_dccr_core.cuh"

namespace sosk {

template <int K>
struct CasDims {
    static constexpr int S = 2 * K;                        // state words of the cascade
    static constexpr int NB = K * (K + 1) / 2;             // 2x2 blocks of a lower block-triangular matrix
    static constexpr int NF = 4 * NB;                      // floats of one packed matrix
    static constexpr int MS = ((NF / 4) & 1) ? NF : NF + 4;  // per-lane stride: conflict-free 128-bit reads
    static constexpr int FULL = S * S;                     // floats of one dense column-major matrix
    static constexpr int P2 = S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;  // S rounded up to a power of 2
    static constexpr int SH = 5 - (P2 == 2 ? 1 : P2 == 4 ? 2 : P2 == 8 ? 3 : 4);  // lane >> SH = word
    // table block copied to shared memory: (M_N)^lane [32][MS], (A_T)^lane [32][MS] (packed),
    // A_C dense column-major; then, in global memory only, A_T dense and (A_T)^(32 w) dense for
    // w = 1..kMaxWin
    static constexpr int TAB = 2 * 32 * MS + FULL;
    static constexpr int TAB_GLOBAL = TAB + (1 + kMaxWin) * FULL;
};

// y = A x for a packed lower block-triangular A (block (s, t), s >= t, at s(s+1)/2 + t, row-major).
template <int K>
__device__ __forceinline__ void packed_mv(const float *__restrict__ A, const float (&x)[2 * K], float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int t = 0; t <= s; ++t) {
            const float4 B = *reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + t));
            y0 = fmaf(B.x, x[2 * t], fmaf(B.y, x[2 * t + 1], y0));
            y1 = fmaf(B.z, x[2 * t], fmaf(B.w, x[2 * t + 1], y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
    }
}

// y = A x with both A (packed) and x in shared memory (x read as word pairs, broadcast).
template <int K>
__device__ __forceinline__ void packed_mv_sx(const float *__restrict__ A, const float *__restrict__ x,
                                             float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = 0.f, y1 = 0.f;
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

// Same with the matrix in the kernel parameter space (compile-time offsets).
template <int K>
__device__ __forceinline__ void packed_mv_param(const float *A, const float (&x)[2 * K], float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int t = 0; t <= s; ++t) {
            const float *B = A + 4 * (s * (s + 1) / 2 + t);
            y0 = fmaf(B[0], x[2 * t], fmaf(B[1], x[2 * t + 1], y0));
            y1 = fmaf(B[2], x[2 * t], fmaf(B[3], x[2 * t + 1], y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
    }
}

// Lane-parallel y = A x for a dense column-major S x S matrix: lane i < S holds x_i and gets y_i.
template <int S>
__device__ __forceinline__ float lane_mv(const float *__restrict__ A, float xi, int lane) {
    float y = 0.f;
    const int row = lane < S ? lane : 0;
#pragma unroll
    for (int j = 0; j < S; ++j) y = fmaf(A[j * S + row], __shfl_sync(0xffffffffu, xi, j), y);
    return y;
}

// Sum t (S words per lane) over the 32 lanes, in place; lane l receives word (l >> SH) of the sum
// (recursive halving: P2/2 + P2/4 + ... + 1 exchanges, then butterflies over the remaining lanes).
template <int S, int P2, int SH>
__device__ __forceinline__ float reduce_scatter(float (&t)[S], int lane) {
#pragma unroll
    for (int h = P2 / 2, off = 16; h >= 1; h /= 2, off /= 2) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float lo = i < S ? t[i] : 0.f;
            const float hi = (h + i) < S ? t[h + i] : 0.f;
            const float send = up ? lo : hi;
            const float keep = up ? hi : lo;
            if (i < S) t[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
#pragma unroll
    for (int off = (1 << SH) / 2; off >= 1; off /= 2) t[0] += __shfl_xor_sync(0xffffffffu, t[0], off);
    return t[0];
}

// Zero-state pass of one group through section s (registers only); the lane's N samples are held as
// N/2 (even, odd) pairs so both divide-and-conquer chains share packed FMAs.
template <int N, bool NORM>
__device__ __forceinline__ void section_zero_state(float2 (&P)[N / 2], const SecCoef &c, int s, float *a_out,
                                                   int lane, bool tail_capture, int m_last, float *zs) {
    constexpr int H = N / 2;
    float xin_m = 0.f, xin_m1 = 0.f;
    if (tail_capture) {
        xin_m = pick_pair<H>(P, m_last);
        xin_m1 = pick_pair<H>(P, m_last > 0 ? m_last - 1 : 0);
    }
    const float xs1 = P[H - 1].y, xs2 = P[H - 1].x;
    SectionPair<N, NORM>::reduce(P, c);
    const float yo = P[H - 1].y, ye = P[H - 1].x;
    float t1 = fmaf(c.b1, xs1, fmaf(c.b2, xs2, -fmaf(c.a1, yo, c.a2 * ye)));
    float t2 = fmaf(c.b2, xs1, -c.a2 * yo);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float u1 = __shfl_up_sync(0xffffffffu, t1, 1 << k);
        const float u2 = __shfl_up_sync(0xffffffffu, t2, 1 << k);
        if (lane >= (1 << k)) {
            t1 = fmaf(c.tn[k][0], u1, fmaf(c.tn[k][1], u2, t1));
            t2 = fmaf(c.tn[k][2], u1, fmaf(c.tn[k][3], u2, t2));
        }
    }
    float zx1 = __shfl_up_sync(0xffffffffu, t1, 1);
    float zx2 = __shfl_up_sync(0xffffffffu, t2, 1);
    if (lane == 0) zx1 = zx2 = 0.f;
    if (lane == 31) {
        a_out[2 * s] = t1;
        a_out[2 * s + 1] = t2;
    }
    SectionPair<N, NORM>::back_substitute(P, c, zx1, zx2);
    if (tail_capture) {
        // transposed direct form II state after the signal's last sample (zero-state part)
        const float ym = pick_pair<H>(P, m_last);
        float f1;
        if (m_last > 0) {
            const float ym1 = pick_pair<H>(P, m_last - 1);
            f1 = c.b1 * xin_m + c.b2 * xin_m1 - c.a1 * ym - c.a2 * ym1;
        } else {
            f1 = c.b1 * xin_m - c.a1 * ym + zx2;
        }
        zs[2 * s] = f1;
        zs[2 * s + 1] = c.b2 * xin_m - c.a2 * ym;
    }
}

// Zero-state pass of one group through the K sections.  Beyond two sections the loop over sections
// stays rolled: one copy of the section code keeps the instruction footprint inside the cache
// (unrolled, orders 8 and 16 stalled on instruction fetch).
template <int K, int N, bool NORM>
__device__ __forceinline__ void cascade_zero_state(float2 (&P)[N / 2], const SecCoef *sec, float *a_out, int lane,
                                                   bool tail_capture, int m_last, float *zs) {
    if constexpr (K <= 2) {
#pragma unroll
        for (int s = 0; s < K; ++s)
            section_zero_state<N, NORM>(P, sec[s], s, a_out, lane, tail_capture, m_last, zs);
    } else {
#pragma unroll 1
        for (int s = 0; s < K; ++s)
            section_zero_state<N, NORM>(P, sec[s], s, a_out, lane, tail_capture, m_last, zs);
    }
}

// The coordinator warp of the cascade-carry kernels (one per block, warp 0: warp schedulers favour
// lower, older warps, and its carry work is on every tile's critical path): for each tile of the
// block it waits for the tile's fold, resolves the tile's incoming 2K-word state by decoupled
// lookback over tiles (Sec. IV-B, Eq. 25 on the cascade state; 32 predecessors per round, the
// first resolved one ends it), posts the tile's resolved carry, and derives the incoming state of
// each of the tile's W groups.  Shared by the single- and double-thread-group kernels.
template <int K, int N, int W>
__device__ __forceinline__ void cascade_coordinator(const CasParams<K, N> &p, int lane, long long budget,
                                                    unsigned long long *bar_local, unsigned long long *bar_zready,
                                                    unsigned long long *bar_ticket, const long long *ring,
                                                    const float *a_buf, float *z_buf, const float *agg,
                                                    const float *sATl, const float *sACd, const float *gATd) {
    using Dm = CasDims<K>;
    constexpr int S = Dm::S, MS = Dm::MS;
    // ------------------------------------------------------------------ coordinator warp
    const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
    // initial state of the signal (scaled domain), word i
    auto zinit = [&](int i) -> float { return p.zi ? p.zi[i] * p.sec[i >> 1].zscale : 0.f; };
    unsigned it = 0;
    for (;;) {
        if (!mbar_wait(&bar_ticket[it & 3], (it >> 2) & 1, budget, p.status)) break;
        const long long cur = ring[it & 3];
        if (cur < 0) break;

        if (!mbar_wait(&bar_local[it & 1], (it >> 1) & 1, budget, p.status)) break;

        unsigned long long *tr = (p.trace && lane == 0 && cur < p.trace_tiles)
                                     ? p.trace + static_cast<size_t>(cur) * kTraceSlots
                                     : nullptr;
        if (tr) {
            unsigned smid;
            asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
            tr[0] = static_cast<unsigned long long>(cur) + 1;
            tr[1] = global_ns();
            tr[11] = smid;
        }
        const float *abuf = a_buf + (it & 1) * W * S;
        const float acc_i = agg[(it & 1) * S + (lane < S ? lane : 0)];  // this lane's word of the tile carry
        float tmp[S];
        if (tr) tr[2] = global_ns();
        unsigned long long *dcur = p.desc + static_cast<size_t>(cur) * S;
        float zi_lane = 0.f;  // word `lane` of the tile's incoming state (lanes < S)
        unsigned n_win = 0, n_wait = 0;
        if (cur == 0) {
            zi_lane = zinit(lane < S ? lane : 0);
        } else {
            // ---- decoupled lookback over tiles, 32 predecessors per round (local carry posted
            // by the folding compute warp)
            const long long t_start = clock64();
            int win = 0;
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
                    st = 2;  // the signal's initial state is the resolved carry of tile -1
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
                    __nanosleep(64);  // leave the issue slots to the computing warps meanwhile
                    continue;
                }
                ++n_win;
                if (lane > j) {
#pragma unroll
                    for (int i = 0; i < S; ++i) v[i] = 0.f;
                }
                // sum over the window of (A_T)^k v_k: each lane applies its own power, then a
                // reduce-scatter leaves word i of the sum in lane i
                packed_mv<K>(sATl + lane * MS, v, tmp);
                float part = reduce_scatter<S, Dm::P2, Dm::SH>(tmp, lane);
                part = __shfl_sync(0xffffffffu, part, (lane < S ? lane : 0) << Dm::SH);
                if (win == 0) {
                    zi_lane += part;
                } else {
                    // (A_T)^(32 win) from the global table (rarely needed)
                    const float *Aw = p.tab + Dm::TAB + win * Dm::FULL;
                    float y = 0.f;
                    const int row = lane < S ? lane : 0;
#pragma unroll
                    for (int jj = 0; jj < S; ++jj) y = fmaf(__ldg(Aw + jj * S + row), __shfl_sync(0xffffffffu, part, jj), y);
                    zi_lane += y;
                }
                if (j < 32) break;
                if (++win > kMaxWin) {  // predecessors too far behind: report and give up
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
            float gl = acc_i;  // A_T Z + tile carry
            {
                const int row = lane < S ? lane : 0;
#pragma unroll
                for (int jj = 0; jj < S; ++jj)
                    gl = fmaf(__ldg(gATd + jj * S + row), __shfl_sync(0xffffffffu, zi_lane, jj), gl);
            }
            if (lane < S) st_relaxed_b64(dcur + lane, pack_word(tagG, gl));
        }
        // incoming state of each group of the tile: Z_0 = Z, Z_{w+1} = A_C Z_w + a_w
        float *zb = z_buf + (it & 1) * W * S;
#pragma unroll 1
        for (int w = 0; w < W; ++w) {
            if (lane < S) zb[w * S + lane] = zi_lane;
            if (w + 1 < W) zi_lane = lane_mv<S>(sACd, zi_lane, lane) + abuf[w * S + (lane < S ? lane : 0)];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_zready[it & 1]);  // one barrier per tile parity
        if (tr) tr[4] = global_ns();
        ++it;
    }
}

template <int K, int N, bool NORM, int W>
__global__ void __launch_bounds__((W + 1) * 32) __maxnreg__(N <= 32 ? 96 : 168) sos_cascade_kernel(const __grid_constant__ CasParams<K, N> p) {
    using Dm = CasDims<K>;
    constexpr int S = Dm::S, NF = Dm::NF, MS = Dm::MS;
    constexpr int P = N + 4;  // padded row pitch (floats): conflict-free 128-bit row access
    constexpr int C = N * kL;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);    // [2][W][32][P]: prefetch X, stash Y
    float *sMl = rows + 2 * W * kL * P;                // [32][MS]: (M_N)^lane
    float *sATl = sMl + kL * MS;                       // [32][MS]: (A_T)^lane
    float *sACd = sATl + kL * MS;                      // A_C dense column-major
    const float *gATd = p.tab + Dm::TAB;               // A_T dense column-major (global, L1-resident)
    float *a_buf = sACd + Dm::FULL;                    // [2][W][S] local carries of the groups
    float *z_buf = a_buf + 2 * W * S;                  // [2][W][S] incoming states of the groups
    float *zs_tail = z_buf + 2 * W * S;                // [S] zero-state final state (last group)
    float *agg = zs_tail + S;                          // [2][S] tile carry under zero incoming state
    __shared__ unsigned long long bar_local[2], bar_zready[2], bar_ticket[4];
    __shared__ long long ring[4];
    __shared__ int fold_count[2];
    __shared__ int tickets_exhausted;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long budget = p.spin_budget;

    {
        const float4 *src = reinterpret_cast<const float4 *>(p.tab);
        float4 *dst = reinterpret_cast<float4 *>(sMl);
        for (int i = threadIdx.x; i < Dm::TAB / 4; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    // Tickets: tile of iteration k in ring[k & 3], posted on bar_ticket[k & 3] (phase (k >> 2) & 1).
    // Thread 0 draws the first two; afterwards the folding warp of iteration k draws k + 2.  Once a
    // draw passes the last tile no further atomics are issued, so a launch consumes exactly
    // n_tiles + gridDim.x tickets.
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
        mbar_init(&bar_local[0], 1);
        mbar_init(&bar_local[1], 1);
        fold_count[0] = fold_count[1] = 0;
        tickets_exhausted = 0;
        mbar_init(&bar_zready[0], 1);
        mbar_init(&bar_zready[1], 1);
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar_ticket[i], 1);
        ring[0] = draw_ticket();
        ring[1] = draw_ticket();
        mbar_arrive(&bar_ticket[0]);
        mbar_arrive(&bar_ticket[1]);
    }
    __syncthreads();

    // Warp 0 coordinates; warps 1..W compute groups 0..W-1 of the tile.
    if (warp == 0) {
        cascade_coordinator<K, N, W>(p, lane, budget, bar_local, bar_zready, bar_ticket, ring, a_buf, z_buf, agg,
                                     sATl, sACd, gATd);
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int w = warp - 1;
    float *X = rows + w * kL * P;
    float *Y = rows + (W + w) * kL * P;
    const bool want_zf = p.zf != nullptr;
    const long long g_last = p.G - 1;
    const long long p_last = p.n - 1 - g_last * C;  // position of the signal's last sample in its group
    const int lane_last = static_cast<int>(p_last / N), m_last = static_cast<int>(p_last % N);

    auto issue_load = [&](long long g) {
        const long long base = g * C;
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

    auto wtrace = [&](long long tile, int slot) {
        if (p.trace && w == 0 && lane == 0 && tile < p.trace_tiles)
            p.trace[static_cast<size_t>(tile) * kTraceSlots + slot] = global_ns();
    };
    auto correct_and_store = [&](long long tile, unsigned jt) -> bool {
        wtrace(tile, 8);
        if (!mbar_wait(&bar_zready[jt & 1], (jt >> 1) & 1, budget, p.status)) return false;
        wtrace(tile, 9);
        const long long g = tile * W + w;
        const float *zb = z_buf + ((jt & 1) * W + w) * S;
        float dz[S];
        packed_mv_sx<K>(sMl + lane * MS, zb, dz);  // lane's incoming cascade state (M_N)^lane Z
        float *row = Y + lane * P;
        float2 dd[S];
#pragma unroll
        for (int j = 0; j < S; ++j) dd[j] = make_float2(dz[j], dz[j]);
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 v = *reinterpret_cast<float4 *>(row + 4 * q);
            float2 e0 = make_float2(v.x, v.y), e1 = make_float2(v.z, v.w);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const float2 *hj = reinterpret_cast<const float2 *>(p.H[j]);
                e0 = __ffma2_rn(hj[2 * q], dd[j], e0);
                e1 = __ffma2_rn(hj[2 * q + 1], dd[j], e1);
            }
            *reinterpret_cast<float4 *>(row + 4 * q) = make_float4(e0.x, e0.y, e1.x, e1.y);
        }
        if (want_zf && g == g_last && lane == lane_last) {
            float Z[S], zt[S];
#pragma unroll
            for (int i = 0; i < S; ++i) Z[i] = zb[i];
            packed_mv_param<K>(p.A_tail, Z, zt);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                p.zf[2 * s] = (zs_tail[2 * s] + zt[2 * s]) * p.sec[s].zscale_inv;
                p.zf[2 * s + 1] = (zs_tail[2 * s + 1] + zt[2 * s + 1]) * p.sec[s].zscale_inv;
            }
        }
        if (g < p.G) {
            const long long base = g * C;
            const long long avail = p.n - base;
            if (avail >= C && p.aligned) {
                fence_proxy_async_smem();
                bulk_store(p.y + base + lane * N, row, N * 4);
                bulk_commit();
                wtrace(tile, 10);
            } else {
                __syncwarp();
#pragma unroll
                for (int j = 0; j < N / 4; ++j) {
                    const int off = 4 * (j * 32 + lane);
                    const float4 v = *reinterpret_cast<const float4 *>(Y + (off / N) * P + (off % N));
                    float *dst = p.y + base + off;
                    if (off + 0 < avail) __stcs(dst + 0, v.x);
                    if (off + 1 < avail) __stcs(dst + 1, v.y);
                    if (off + 2 < avail) __stcs(dst + 2, v.z);
                    if (off + 3 < avail) __stcs(dst + 3, v.w);
                }
            }
        }
        return true;
    };

    if (!mbar_wait(&bar_ticket[0], 0, budget, p.status)) return;
    long long tile = ring[0];
    if (tile < 0) return;
    issue_load(tile * W + w);
    unsigned it = 0;
    long long prev = -1;
    bool ok = true;
    for (;;) {
        const long long g = tile * W + w;
        cp_async_wait_all();
        __syncwarp();
        float2 r[N / 2];
#pragma unroll
        for (int j = 0; j < N / 4; ++j) {
            const float4 v = *reinterpret_cast<const float4 *>(X + lane * P + 4 * j);
            r[2 * j + 0] = make_float2(v.x, v.y);
            r[2 * j + 1] = make_float2(v.z, v.w);
        }
        if (NORM) {
            const float2 gg = make_float2(p.gain, p.gain);
#pragma unroll
            for (int j = 0; j < N / 2; ++j) r[j] = __fmul2_rn(r[j], gg);
        }
        __syncwarp();
        if (!mbar_wait(&bar_ticket[(it + 1) & 3], ((it + 1) >> 2) & 1, budget, p.status)) {
            ok = false;
            break;
        }
        const long long next = ring[(it + 1) & 3];
        if (next >= 0) issue_load(next * W + w);

        wtrace(tile, 6);
        cascade_zero_state<K, N, NORM>(r, p.sec, a_buf + ((it & 1) * W + w) * S, lane,
                                       want_zf && g == g_last && lane == lane_last, m_last, zs_tail);
        wtrace(tile, 7);
        {
            // The last warp of the tile to finish its pass folds the groups' local carries into the
            // tile's (c = a_0; c = A_C c + a_w) and posts it at once, so successors never wait on
            // this block's coordinator for it.
            __syncwarp();
            int old = 0;
            if (lane == 0) {
                __threadfence_block();
                old = atomicAdd(&fold_count[it & 1], 1);
            }
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == W - 1) {
                __threadfence_block();
                const float *ab = a_buf + (it & 1) * W * S;
                const int li = lane < S ? lane : 0;
                float c = ab[li];
#pragma unroll 1
                for (int v = 1; v < W; ++v) c = lane_mv<S>(sACd, c, lane) + ab[v * S + li];
                if (tile > 0 && lane < S)
                    st_relaxed_b64(p.desc + static_cast<size_t>(tile) * S + lane,
                                   pack_word((p.epoch << 2) | 1u, c));
                if (lane < S) agg[(it & 1) * S + lane] = c;
                if (lane == 0) {
                    fold_count[it & 1] = 0;
                    ring[(it + 2) & 3] = draw_ticket();
                    mbar_arrive(&bar_ticket[(it + 2) & 3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_local[it & 1]);
            }
        }

        if (prev >= 0 && !correct_and_store(prev, it - 1)) {
            ok = false;
            break;
        }
        bulk_wait_read0();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < N / 4; ++j)
            *reinterpret_cast<float4 *>(Y + lane * P + 4 * j) =
                make_float4(r[2 * j].x, r[2 * j].y, r[2 * j + 1].x, r[2 * j + 1].y);
        __syncwarp();
        prev = tile;
        if (next < 0) break;
        tile = next;
        ++it;
    }
    if (ok) correct_and_store(prev, it);
    bulk_wait0();
}

}  // namespace sosk
