// Multi-signal persistent kernel, sm_103a: many signals of uneven length, one section count K,
// in one launch over a global queue of (signal, tile) work items.
//
// The work of every signal is cut into tiles of W = kBatchW groups of C = 32 N samples
// (N = kBatchN); the tiles of all signals of the launch form one queue, drawn in ascending order
// from a ticket counter (Sec. IV-A), so that tile t's predecessors within its signal are held by
// running or finished blocks.  Each tile is filtered as by the single-signal cascade kernel
// (sosfilt_cascade.cuh): a zero-state pass per group (divide-and-conquer cyclic reduction per
// section, Sec. II-E, lanes scanned inside the warp), a coordinator warp that folds the groups'
// local carries, resolves the tile's incoming 2K-word state by decoupled lookback (Sec. IV-B,
// Eq. 25 on the cascade state) and derives the groups' incoming states, and the homogeneous
// correction of Eq. 24 applied once for the cascade.  What changes is that lookback chains are
// kept per signal (a chain ends at its signal's first tile, whose incoming state is the signal's
// initial state) and that every per-signal quantity (pointers, length, section tables, output
// basis, transition tables) comes from the signal's descriptor in global memory.
#pragma once
#include "sosfilt_cascade.cuh"

namespace sosk {

// y = A x, A packed lower block-triangular in global memory, x in shared memory (broadcast pairs).
template <int K>
__device__ __forceinline__ void packed_mv_gs(const float *__restrict__ A, const float *__restrict__ x,
                                             float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int t = 0; t <= s; ++t) {
            const float4 B = __ldg(reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + t)));
            const float2 xt = *reinterpret_cast<const float2 *>(x + 2 * t);
            y0 = fmaf(B.x, xt.x, fmaf(B.y, xt.y, y0));
            y1 = fmaf(B.z, xt.x, fmaf(B.w, xt.y, y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
    }
}

// Same with x in registers.
template <int K>
__device__ __forceinline__ void packed_mv_gr(const float *__restrict__ A, const float (&x)[2 * K],
                                             float (&y)[2 * K]) {
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
    }
}

// Lane-parallel y = A x for a dense column-major S x S matrix in global memory.
template <int S>
__device__ __forceinline__ float lane_mv_g(const float *__restrict__ A, float xi, int lane) {
    float y = 0.f;
    const int row = lane < S ? lane : 0;
#pragma unroll
    for (int j = 0; j < S; ++j) y = fmaf(__ldg(A + j * S + row), __shfl_sync(0xffffffffu, xi, j), y);
    return y;
}

template <int K, bool NORM>
__global__ void __maxnreg__(96) sos_batch_kernel(const __grid_constant__ BatchParams<K> p) {
    using Dm = CasDims<K>;
    constexpr int S = Dm::S, MS = Dm::MS, N = kBatchN, W = kBatchW;
    constexpr int P = N + 4;  // padded row pitch (floats): conflict-free 128-bit row access
    constexpr int C = N * kL;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);  // [2][W][32][P]: prefetch X, stash Y
    float *a_buf = rows + 2 * W * kL * P;            // [2][W][S] local carries of the groups
    float *z_buf = a_buf + 2 * W * S;                // [2][W][S] incoming states of the groups
    float *zs_tail = z_buf + 2 * W * S;              // [2][S] zero-state final state (a signal's last group)
    float *agg = zs_tail + 2 * S;                    // [2][S] tile carry under zero incoming state
    __shared__ unsigned long long bar_local[2], bar_zready[2], bar_ticket[4];
    __shared__ long long ring[4];
    __shared__ int ring_sig[4];
    __shared__ int fold_count[2];
    __shared__ int tickets_exhausted;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long budget = p.spin_budget;

    // Tickets: tile of iteration k in ring[k & 3] with its signal in ring_sig[k & 3], posted on
    // bar_ticket[k & 3] (phase (k >> 2) & 1).  Thread 0 draws the first two; afterwards the folding
    // warp of iteration k draws k + 2.
    auto draw_ticket = [&](int slot) {
        long long t = -1;
        if (!tickets_exhausted) {
            t = static_cast<long long>(atomicAdd(p.ticket, 1ULL) - p.ticket_base);
            if (t >= p.n_tiles) {
                tickets_exhausted = 1;
                t = -1;
            }
        }
        ring[slot] = t;
        ring_sig[slot] = t >= 0 ? __ldg(p.tile_sig + t) : -1;
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar_local[0], 1);
        mbar_init(&bar_local[1], 1);
        mbar_init(&bar_zready[0], 1);
        mbar_init(&bar_zready[1], 1);
        fold_count[0] = fold_count[1] = 0;
        tickets_exhausted = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar_ticket[i], 1);
        draw_ticket(0);
        draw_ticket(1);
        mbar_arrive(&bar_ticket[0]);
        mbar_arrive(&bar_ticket[1]);
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------------ coordinator warp
        const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
        unsigned it = 0;
        for (;;) {
            if (!mbar_wait(&bar_ticket[it & 3], (it >> 2) & 1, budget, p.status)) break;
            const long long cur = ring[it & 3];
            if (cur < 0) break;
            const BatchSig *sg = p.sigs + ring_sig[it & 3];
            const long long tile0 = sg->tile0;
            const float *tab = sg->tab;
            const float *gATd = tab + Dm::TAB;
            const float *zi = sg->zi;
            const SecCoef *sec = sg->sec;
            // initial state of the signal (scaled domain), word i
            auto zinit = [&](int i) -> float { return zi ? zi[i] * sec[i >> 1].zscale : 0.f; };
            if (!mbar_wait(&bar_local[it & 1], (it >> 1) & 1, budget, p.status)) break;
            const float *abuf = a_buf + (it & 1) * W * S;
            const float acc_i = agg[(it & 1) * S + (lane < S ? lane : 0)];
            float tmp[S];
            unsigned long long *dcur = p.desc + static_cast<size_t>(cur) * S;
            float zi_lane = 0.f;
            if (cur == tile0) {
                zi_lane = zinit(lane < S ? lane : 0);
            } else {
                // decoupled lookback over the signal's tiles, 32 predecessors per round
                const long long t_start = clock64();
                int win = 0;
                for (;;) {
                    const long long pred = cur - 1 - 32LL * win - lane;
                    float v[S];
                    int st;
                    if (pred >= tile0) {
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
                        st = 2;  // the signal's initial state is the resolved carry of its tile -1
#pragma unroll
                        for (int i = 0; i < S; ++i) v[i] = (pred == tile0 - 1) ? zinit(i) : 0.f;
                    }
                    const unsigned glob = __ballot_sync(0xffffffffu, st == 2);
                    const unsigned inv = __ballot_sync(0xffffffffu, st == 0);
                    const int j = glob ? __ffs(glob) - 1 : 32;
                    const unsigned need = (j >= 31) ? 0xffffffffu : ((2u << j) - 1u);
                    if (inv & need) {
                        if (__any_sync(0xffffffffu, (clock64() - t_start) > budget)) {
                            if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    if (lane > j) {
#pragma unroll
                        for (int i = 0; i < S; ++i) v[i] = 0.f;
                    }
                    // sum over the window of (A_T)^k v_k (lane's own power), reduce-scattered
                    packed_mv_gr<K>(tab + (32 + lane) * MS, v, tmp);
                    float part = reduce_scatter<S, Dm::P2, Dm::SH>(tmp, lane);
                    part = __shfl_sync(0xffffffffu, part, (lane < S ? lane : 0) << Dm::SH);
                    if (win == 0) {
                        zi_lane += part;
                    } else {
                        const float *Aw = gATd + win * Dm::FULL;
                        zi_lane += lane_mv_g<S>(Aw, part, lane);
                    }
                    if (j < 32) break;
                    if (++win > kMaxWin) {
                        if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                        break;
                    }
                }
            }
            if (cur + 1 < p.n_tiles) {
                // the resolved carry A_T Z + tile carry (read by the signal's next tile only)
                const float gl = lane_mv_g<S>(gATd, zi_lane, lane) + acc_i;
                if (lane < S) st_relaxed_b64(dcur + lane, pack_word(tagG, gl));
            }
            // incoming state of each group of the tile: Z_0 = Z, Z_{w+1} = A_C Z_w + a_w
            const float *ACd = tab + 64 * MS;
            float *zb = z_buf + (it & 1) * W * S;
#pragma unroll 1
            for (int w = 0; w < W; ++w) {
                if (lane < S) zb[w * S + lane] = zi_lane;
                if (w + 1 < W) zi_lane = lane_mv_g<S>(ACd, zi_lane, lane) + abuf[w * S + (lane < S ? lane : 0)];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_zready[it & 1]);  // one barrier per tile parity
            ++it;
        }
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int w = warp - 1;
    float *X = rows + w * kL * P;
    float *Y = rows + (W + w) * kL * P;

    // group w of global tile `tile` belongs to signal sg; its index within the signal is
    // (tile - tile0) W + w
    auto issue_load = [&](long long tile, const BatchSig *sg) {
        const long long g = (tile - sg->tile0) * W + w;
        const long long base = g * C;
        const long long avail = sg->n - base;
        const float *x = sg->x;
        if (avail >= C && sg->aligned) {
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const int off = 4 * (j * 32 + lane);
                cp_async16(X + (off / N) * P + (off % N), x + base + off);
            }
            cp_async_commit();
        } else {
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const int off = 4 * (j * 32 + lane);
                float4 v;
                v.x = (off + 0 < avail) ? __ldcs(x + base + off + 0) : 0.f;
                v.y = (off + 1 < avail) ? __ldcs(x + base + off + 1) : 0.f;
                v.z = (off + 2 < avail) ? __ldcs(x + base + off + 2) : 0.f;
                v.w = (off + 3 < avail) ? __ldcs(x + base + off + 3) : 0.f;
                *reinterpret_cast<float4 *>(X + (off / N) * P + (off % N)) = v;
            }
        }
    };

    auto correct_and_store = [&](long long tile, int sig, unsigned jt) -> bool {
        if (!mbar_wait(&bar_zready[jt & 1], (jt >> 1) & 1, budget, p.status)) return false;
        const BatchSig *sg = p.sigs + sig;
        const long long g = (tile - sg->tile0) * W + w;
        const long long G = sg->G;
        const float *zb = z_buf + ((jt & 1) * W + w) * S;
        float dz[S];
        packed_mv_gs<K>(sg->tab + lane * MS, zb, dz);  // lane's incoming cascade state (M_N)^lane Z
        float *row = Y + lane * P;
        const float2 *H = reinterpret_cast<const float2 *>(sg->H);
        float2 dd[S];
#pragma unroll
        for (int j = 0; j < S; ++j) dd[j] = make_float2(dz[j], dz[j]);
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 v = *reinterpret_cast<float4 *>(row + 4 * q);
            float2 e0 = make_float2(v.x, v.y), e1 = make_float2(v.z, v.w);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                e0 = __ffma2_rn(__ldg(H + j * (N / 2) + 2 * q), dd[j], e0);
                e1 = __ffma2_rn(__ldg(H + j * (N / 2) + 2 * q + 1), dd[j], e1);
            }
            *reinterpret_cast<float4 *>(row + 4 * q) = make_float4(e0.x, e0.y, e1.x, e1.y);
        }
        if (g == G - 1 && sg->zf) {
            const long long p_last = sg->n - 1 - (G - 1) * C;
            if (lane == static_cast<int>(p_last / N)) {
                // the lane's incoming state from Z is dz = (M_N)^lane Z; carried over the lane's
                // samples up to the last one: M1^(m_last + 1) dz
                float zt[S];
                packed_mv_gr<K>(sg->Mm + static_cast<int>(p_last % N) * Dm::NF, dz, zt);
                const float *zs = zs_tail + (jt & 1) * S;
                float *zf = sg->zf;
                const SecCoef *sec = sg->sec;
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    const float inv = sec[s].zscale_inv;
                    zf[2 * s] = (zs[2 * s] + zt[2 * s]) * inv;
                    zf[2 * s + 1] = (zs[2 * s + 1] + zt[2 * s + 1]) * inv;
                }
            }
        }
        if (g < G) {
            const long long base = g * C;
            const long long avail = sg->n - base;
            float *y = sg->y;
            if (avail >= C && sg->aligned) {
                fence_proxy_async_smem();
                bulk_store(y + base + lane * N, row, N * 4);
                bulk_commit();
            } else {
                __syncwarp();
#pragma unroll
                for (int j = 0; j < N / 4; ++j) {
                    const int off = 4 * (j * 32 + lane);
                    const float4 v = *reinterpret_cast<const float4 *>(Y + (off / N) * P + (off % N));
                    if (off + 0 < avail) __stcs(y + base + off + 0, v.x);
                    if (off + 1 < avail) __stcs(y + base + off + 1, v.y);
                    if (off + 2 < avail) __stcs(y + base + off + 2, v.z);
                    if (off + 3 < avail) __stcs(y + base + off + 3, v.w);
                }
            }
        }
        return true;
    };

    if (!mbar_wait(&bar_ticket[0], 0, budget, p.status)) return;
    long long tile = ring[0];
    int sig = ring_sig[0];
    if (tile < 0) return;
    issue_load(tile, p.sigs + sig);
    unsigned it = 0;
    long long prev = -1;
    int prev_sig = -1;
    bool ok = true;
    for (;;) {
        const BatchSig *sg = p.sigs + sig;
        const long long g = (tile - sg->tile0) * W + w;
        const long long G = sg->G;
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
            const float gn = sg->gain;
            const float2 gg = make_float2(gn, gn);
#pragma unroll
            for (int j = 0; j < N / 2; ++j) r[j] = __fmul2_rn(r[j], gg);
        }
        __syncwarp();
        if (!mbar_wait(&bar_ticket[(it + 1) & 3], ((it + 1) >> 2) & 1, budget, p.status)) {
            ok = false;
            break;
        }
        const long long next = ring[(it + 1) & 3];
        const int next_sig = ring_sig[(it + 1) & 3];
        if (next >= 0) issue_load(next, p.sigs + next_sig);

        {
            const bool cap = (g == G - 1) && sg->zf != nullptr;
            const long long p_last = sg->n - 1 - (G - 1) * C;
            cascade_zero_state<K, N, NORM>(r, sg->sec, a_buf + ((it & 1) * W + w) * S, lane,
                                           cap && lane == static_cast<int>(p_last / N), static_cast<int>(p_last % N),
                                           zs_tail + (it & 1) * S);
        }
        {
            // the last warp of the tile to finish folds the groups' local carries (c = a_0;
            // c = A_C c + a_w), posts the tile's carry and draws the ticket two tiles ahead
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
                const float *ACd = sg->tab + 64 * MS;
                const int li = lane < S ? lane : 0;
                float c = ab[li];
#pragma unroll 1
                for (int v = 1; v < W; ++v) c = lane_mv_g<S>(ACd, c, lane) + ab[v * S + li];
                if (tile > sg->tile0 && lane < S)
                    st_relaxed_b64(p.desc + static_cast<size_t>(tile) * S + lane, pack_word((p.epoch << 2) | 1u, c));
                if (lane < S) agg[(it & 1) * S + lane] = c;
                if (lane == 0) {
                    fold_count[it & 1] = 0;
                    draw_ticket((it + 2) & 3);
                    mbar_arrive(&bar_ticket[(it + 2) & 3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_local[it & 1]);
            }
        }

        if (prev >= 0 && !correct_and_store(prev, prev_sig, it - 1)) {
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
        prev_sig = sig;
        if (next < 0) break;
        tile = next;
        sig = next_sig;
        ++it;
    }
    if (ok) correct_and_store(prev, prev_sig, it);
    bulk_wait0();
}

template <int K>
constexpr size_t batch_smem_bytes() {
    using Dm = CasDims<K>;
    return sizeof(float) * (static_cast<size_t>(2) * kBatchW * kL * (kBatchN + 4) + 4 * kBatchW * Dm::S + 4 * Dm::S);
}

}  // namespace sosk
