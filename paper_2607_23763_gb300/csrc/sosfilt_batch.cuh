// Multi-signal persistent kernel, sm_103a: many signals of uneven length, one section count K,
// in one launch over a global queue of (signal, tile) work items.
//
// The work of every signal is cut into tiles of W = kBatchW groups of C = 32 N samples
// (N = 64, or N = 32 for the short geometry); the tiles of all signals of a class form one queue, drawn in ascending order
// from a ticket counter (Sec. IV-A), so that tile t's predecessors within its signal are held by
// running or finished blocks.  Each tile is filtered as by the single-signal PH kernel
// (sosfilt_lane.cuh): a skewed particular pass per lane in direct-form-I order (Sec. II-C), the
// cascade lane scan, a coordinator warp that folds the groups' local carries, resolves the tile's incoming
// 2K-word state by decoupled lookback (Sec. IV-B, Eq. 25 on the cascade state) and derives the
// groups' incoming states, and the homogeneous correction of Eq. 24 applied once for the cascade.
// What changes is that lookback chains are kept per signal (the anchors count from the signal's
// first tile, whose incoming state is the signal's initial state); that every per-signal quantity
// (pointers, length, section constants, transition tables, output basis) comes from the signal's
// descriptor in global memory, the recurrence coefficients going to registers once per tile; and
// that the next tile's input is staged by cp.async into a third row buffer of the warp.
#pragma once
#include "sosfilt_lane.cuh"

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

// Row `lane` of a dense column-major S x S matrix in global memory, into registers (one latency
// for a chain of products with the same matrix).
template <int S>
__device__ __forceinline__ void load_row_g(const float *__restrict__ A, int lane, float (&r)[S]) {
    const int row = lane < S ? lane : 0;
#pragma unroll
    for (int j = 0; j < S; ++j) r[j] = __ldg(A + j * S + row);
}

// Lane-parallel y = A x with lane i holding row i of A (load_row_g) and x_i.
template <int S>
__device__ __forceinline__ float lane_mv_rows(const float (&r)[S], float xi) {
    float y = 0.f;
#pragma unroll
    for (int j = 0; j < S; ++j) y = fmaf(r[j], __shfl_sync(0xffffffffu, xi, j), y);
    return y;
}

// One block's share of a class of the batch (signals of K sections with the same b0 handling and
// tile geometry, N samples per lane): the block draws tiles from the class's ticket counter until
// the class is exhausted, then returns.
template <int K, bool NORM, int N>
__device__ __forceinline__ void batch_body(const BatchParams<K> &p, float4 *smem4) {
    using Dm = LaneDims<K, N, kBatchW>;
    constexpr int S = Dm::S, MS = Dm::MS, W = kBatchW, RSP = Dm::RSP;
    // the correction takes four consecutive samples of a row per lane and step: CH chunks per row,
    // RPS rows per step
    constexpr int CH = N / 4, RPS = 32 / CH;
    static_assert(CH == Dm::LQ && CH * RPS == 32, "batch tile geometry");
    constexpr int P = N + 4;  // padded row pitch (floats): conflict-free 128-bit row access
    constexpr int C = N * kL;
    constexpr int SZ = ((S + 3) / 4) * 4;
    float *rows = reinterpret_cast<float *>(smem4);  // [W][3][32][P]: three row buffers per warp
    float *rowst = rows + W * 3 * kL * P;            // [W][32][RSP] rows' true incoming states
    float *a_buf = rowst + W * kL * RSP;             // [2][W][S] local carries of the groups
    float *z_buf = a_buf + 2 * W * S;                // [2][W][S] incoming states of the groups
    float *agg = z_buf + 2 * W * S;                  // [2][S] tile carry under zero incoming state
    // [2][W][SZ] lane-local state after a signal's last sample, per slot and warp: a warp overwrites
    // only its own capture, after its own correction has read it (another warp may run two tiles
    // ahead, into the same slot, before this one corrects)
    float *zs_tail = agg + 2 * S;
    __shared__ unsigned long long bar_local[2], bar_zready[2], bar_ticket[8];
    __shared__ long long ring[8];
    __shared__ int ring_sig[8];
    __shared__ int fold_count[2];
    __shared__ int tickets_exhausted;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long budget = p.spin_budget;

    // Tickets: tile of iteration k in ring[k & 7] with its signal in ring_sig[k & 7], posted on
    // bar_ticket[k & 7] (phase (k >> 3) & 1).  Thread 0 draws the first two; afterwards the folding
    // warp of iteration k draws k + 2 (two ahead, not three: tiles are then numbered closer to when
    // blocks reach them, and a tile's predecessors fold closer to it -- 6 % faster on the batched
    // mix), which still leaves a tile's input staged one iteration ahead.
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
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_local[i], 1);
            mbar_init(&bar_zready[i], 1);
            fold_count[i] = 0;
        }
        tickets_exhausted = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) mbar_init(&bar_ticket[i], 1);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            draw_ticket(i);
            mbar_arrive(&bar_ticket[i]);
        }
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------------ coordinator warp
        const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
        unsigned it = 0;
        for (;;) {
            const unsigned slot = it & 1;
            if (!mbar_wait(&bar_ticket[it & 7], (it >> 3) & 1, budget, p.status)) break;
            const long long cur = ring[it & 7];
            if (cur < 0) break;
            const BatchSig *sg = p.sigs + ring_sig[it & 7];
            const long long tile0 = sg->tile0;
            const float *tab = sg->tab;
            const float *zi = sg->zi;
            const LaneSec *sec = sg->sec;
            // initial state of the signal (scaled domain), word i
            auto zinit = [&](int i) -> float { return zi ? zi[i] * __ldg(&sec[i >> 1].zscale) : 0.f; };
            // rows of A_C and A_T for this lane, loaded while the tile's groups are still running
            float acr[S], atr[S];
            load_row_g<S>(tab + Dm::OFF_AC, lane, acr);
            load_row_g<S>(tab + Dm::OFF_AT, lane, atr);
            if (!mbar_wait(&bar_local[slot], (it >> 1) & 1, budget, p.status)) break;
            const float *abuf = a_buf + slot * W * S;
            const float acc_i = agg[slot * S + (lane < S ? lane : 0)];
            float tmp[S];
            unsigned long long *dcur = p.desc + static_cast<size_t>(cur) * 2 * S + S;  // resolved slot
            float zi_lane = 0.f;
            if (cur == tile0) {
                zi_lane = zinit(lane < S ? lane : 0);
            } else {
                // decoupled lookback over the signal's tiles with a fixed composition: the resolved
                // carry of the anchor (the signal's last tile at a multiple of 32 from its first) and
                // the local carries after it, so that outputs are reproducible bit for bit
                const long long a = tile0 + ((cur - 1 - tile0) / 32) * 32;
                const int ja = static_cast<int>(cur - 1 - a);  // the anchor's lane
                const long long pred = cur - 1 - lane;
                const long long t_start = clock64();
                float v[S];
                for (;;) {
                    bool ok = true;
                    if (lane <= ja) {
                        const unsigned want = lane == ja ? tagG : tagL;
                        const unsigned long long *dp = p.desc + static_cast<size_t>(pred) * 2 * S + (lane == ja ? S : 0);
#pragma unroll
                        for (int q = 0; q < S; q += 2) {
                            unsigned long long x0, x1;
                            ld_relaxed_v2(dp + q, x0, x1);
                            ok = ok && static_cast<unsigned>(x0 >> 32) == want && static_cast<unsigned>(x1 >> 32) == want;
                            v[q] = __uint_as_float(static_cast<unsigned>(x0));
                            v[q + 1] = __uint_as_float(static_cast<unsigned>(x1));
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < S; ++q) v[q] = 0.f;
                    }
                    if (__all_sync(0xffffffffu, ok)) break;
                    if (__any_sync(0xffffffffu, (clock64() - t_start) > budget)) {
                        if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
                // sum over the predecessors of (A_T)^k v_k (lane's own power), reduce-scattered
                packed_mv_gr<K>(tab + Dm::OFF_ATL + lane * MS, v, tmp);
                const float part = reduce_scatter<S, Dm::P2, Dm::SH>(tmp, lane);
                zi_lane = __shfl_sync(0xffffffffu, part, (lane < S ? lane : 0) << Dm::SH);
            }
            if (((cur - tile0) & 31) == 0 && cur + 1 < p.n_tiles) {
                // the resolved carry A_T Z + tile carry (read only at the signal's anchor tiles)
                const float gl = lane_mv_rows<S>(atr, zi_lane) + acc_i;
                if (lane < S) st_relaxed_b64(dcur + lane, pack_word(tagG, gl));
            }
            // incoming state of each group of the tile: Z_0 = Z, Z_{v+1} = A_C Z_v + a_v
            float *zb = z_buf + slot * W * S;
#pragma unroll 1
            for (int v = 0; v < W; ++v) {
                if (lane < S) zb[v * S + lane] = zi_lane;
                if (v + 1 < W) zi_lane = lane_mv_rows<S>(acr, zi_lane) + abuf[v * S + (lane < S ? lane : 0)];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_zready[slot]);  // one barrier per tile parity
            ++it;
        }
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int w = warp - 1;
    float *B0 = rows + w * 3 * kL * P;  // the warp's three row buffers
    float *RS = rowst + w * kL * RSP;

    // group w of global tile `tile` belongs to signal sg; its index within the signal is
    // (tile - tile0) W + w
    auto issue_load = [&](long long tile, const BatchSig *sg, float *X) {
        const long long g = (tile - sg->tile0) * W + w;
        const long long base = g * C;
        const long long avail = sg->n - base;
        const float *x = sg->x;
        if (avail <= 0) return;  // a group past the signal's end is not filtered (see below)
        // every copy is asynchronous, so no warp waits on its loads here: the group's ragged end and
        // whatever lies past the signal are zero-filled by the copies themselves (no global read;
        // their source address is the signal's first sample, which always exists)
        if (sg->aligned) {
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int off = 4 * (j * 32 + lane);
                const long long rem = avail - off;
                const unsigned bytes = rem >= 4 ? 16u : rem > 0 ? static_cast<unsigned>(4 * rem) : 0u;
                cp_async16_zfill(X + (off / N) * P + (off % N), bytes ? x + base + off : x, bytes);
            }
        } else {
            // a signal that does not start on a 16-byte boundary: one 4-byte copy per sample
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int off = 4 * (j * 32 + lane);
                float *dst = X + (off / N) * P + (off % N);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool in = off + q < avail;
                    cp_async4_zfill(dst + q, in ? x + base + off + q : x, in ? 4u : 0u);
                }
            }
        }
        cp_async_commit();
    };

    // Correction of the tile of iteration jt (signal sig), whose particular output is in buffer Y
    // and whose lanes' scan states are Sl: rows' true states to shared memory, then four samples per
    // lane across the rows, stored straight to y.
    auto correct_and_store = [&](long long tile, int sig, unsigned jt, const float *Y, const float (&Sl)[S]) -> bool {
        const unsigned slot = jt & 1;
        if (!mbar_wait(&bar_zready[slot], (jt >> 1) & 1, budget, p.status)) return false;
        const BatchSig *sg = p.sigs + sig;
        const long long g = (tile - sg->tile0) * W + w;
        const long long G = sg->G;
        float st[S];
        packed_mv_gs<K>(sg->tab + lane * MS, z_buf + (slot * W + w) * S, st);  // (M_N)^lane Z
#pragma unroll
        for (int j = 0; j < S; ++j) st[j] += Sl[j];
        if (g == G - 1 && sg->zf) {
            const long long p_last = sg->n - 1 - (G - 1) * C;
            if (lane == static_cast<int>(p_last / N)) {
                // final state: lane-local state after the last sample plus the transition of the
                // lane's incoming state over the samples up to it, M1^(m_last + 1) st
                float zt[S];
                packed_mv_gr<K>(sg->Mm + static_cast<int>(p_last % N) * Dm::NF, st, zt);
                const float *zs = zs_tail + (slot * W + w) * SZ;
                float *zf = sg->zf;
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    const float inv = __ldg(&sg->sec[s].zscale_inv);
                    zf[2 * s] = (zs[2 * s] + zt[2 * s]) * inv;
                    zf[2 * s + 1] = (zs[2 * s + 1] + zt[2 * s + 1]) * inv;
                }
            }
        }
        if (g >= G) return true;
#pragma unroll
        for (int j = 0; j < S; j += 2)
            *reinterpret_cast<float2 *>(RS + lane * RSP + j) = make_float2(st[j], st[j + 1]);
        __syncwarp();
        const int c = lane % CH, rsub = lane / CH;
        const float4 *H4 = reinterpret_cast<const float4 *>(sg->tab + Dm::OFF_H);
        float4 h[S];
#pragma unroll
        for (int j = 0; j < S; ++j) h[j] = __ldg(H4 + j * CH + c);
        const long long base = g * C;
        const long long avail = sg->n - base;
        const bool full = avail >= C && sg->aligned;
        float *y = sg->y;
#pragma unroll 2
        for (int r0 = 0; r0 < kL; r0 += RPS) {
            const int r = r0 + rsub;
            float4 v = *reinterpret_cast<const float4 *>(Y + r * P + 4 * c);
            const float *sr = RS + r * RSP;
#pragma unroll
            for (int j = 0; j < S; j += 2) {
                const float2 z = *reinterpret_cast<const float2 *>(sr + j);
                v.x = fmaf(h[j].x, z.x, fmaf(h[j + 1].x, z.y, v.x));
                v.y = fmaf(h[j].y, z.x, fmaf(h[j + 1].y, z.y, v.y));
                v.z = fmaf(h[j].z, z.x, fmaf(h[j + 1].z, z.y, v.z));
                v.w = fmaf(h[j].w, z.x, fmaf(h[j + 1].w, z.y, v.w));
            }
            const int off = r * N + 4 * c;
            if (full) {
                __stcs(reinterpret_cast<float4 *>(y + base + off), v);
            } else {
                float *dst = y + base + off;
                if (off + 0 < avail) __stcs(dst + 0, v.x);
                if (off + 1 < avail) __stcs(dst + 1, v.y);
                if (off + 2 < avail) __stcs(dst + 2, v.z);
                if (off + 3 < avail) __stcs(dst + 3, v.w);
            }
        }
        __syncwarp();
        return true;
    };

    if (!mbar_wait(&bar_ticket[0], 0, budget, p.status)) return;
    long long tile = ring[0];
    int sig = ring_sig[0];
    if (tile < 0) return;
    issue_load(tile, p.sigs + sig, B0);
    unsigned it = 0;
    long long prev = -1;
    int prev_sig = -1;
    float Sprev[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Sprev[j] = 0.f;
    bool ok = true;
    int cur_buf = 0;  // buffer of this iteration's tile; the next tile goes to (cur_buf + 1) % 3
    for (;;) {
        const unsigned slot = it & 1;
        const BatchSig *sg = p.sigs + sig;
        const long long g = (tile - sg->tile0) * W + w;
        const long long G = sg->G;
        float *X = B0 + cur_buf * kL * P;
        const int nxt_buf = cur_buf == 2 ? 0 : cur_buf + 1;
        const int prv_buf = cur_buf == 0 ? 2 : cur_buf - 1;
        cp_async_wait_all();
        __syncwarp();
        if (!mbar_wait(&bar_ticket[(it + 1) & 7], ((it + 1) >> 3) & 1, budget, p.status)) {
            ok = false;
            break;
        }
        const long long next = ring[(it + 1) & 7];
        const int next_sig = ring_sig[(it + 1) & 7];
        if (next >= 0) issue_load(next, p.sigs + next_sig, B0 + nxt_buf * kL * P);

        float t[S], Sl[S];
        if (g < G) {
            const RegSecs<K, NORM> cs(sg->sec, sg->MX);
            const long long p_last = sg->n - 1 - (G - 1) * C;
            if (g == G - 1 && sg->zf)
                lane_particular<K, N, NORM, true>(cs, X + lane * P, sg->gain, t, static_cast<int>(p_last % N),
                                                  lane == static_cast<int>(p_last / N), zs_tail + (slot * W + w) * SZ);
            else
                lane_particular<K, N, NORM, false>(cs, X + lane * P, sg->gain, t, 0, false, nullptr);
            lane_scan<K>(cs, t, Sl, a_buf + (slot * W + w) * S, lane);
        } else {
            // a group past the signal's end (the signal's last tile is not full): nothing to filter,
            // and its local carry, zero, enters the fold as the carry of zero input
#pragma unroll
            for (int j = 0; j < S; ++j) Sl[j] = 0.f;
            if (lane < S) a_buf[(slot * W + w) * S + lane] = 0.f;
        }
        {
            // the last warp of the tile to finish folds the groups' local carries (c = a_0;
            // c = A_C c + a_v), posts the tile's carry and draws the ticket two tiles ahead
            __syncwarp();
            int old = 0;
            if (lane == 0) {
                __threadfence_block();
                old = atomicAdd(&fold_count[slot], 1);
            }
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == W - 1) {
                __threadfence_block();
                const float *ab = a_buf + slot * W * S;
                float acr[S];
                load_row_g<S>(sg->tab + Dm::OFF_AC, lane, acr);
                const int li = lane < S ? lane : 0;
                float c = ab[li];
#pragma unroll 1
                for (int v = 1; v < W; ++v) c = lane_mv_rows<S>(acr, c) + ab[v * S + li];
                if (tile > sg->tile0 && lane < S)
                    st_relaxed_b64(p.desc + static_cast<size_t>(tile) * 2 * S + lane, pack_word((p.epoch << 2) | 1u, c));
                if (lane < S) agg[slot * S + lane] = c;
                if (lane == 0) {
                    fold_count[slot] = 0;
                    draw_ticket((it + 2) & 7);
                    mbar_arrive(&bar_ticket[(it + 2) & 7]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_local[slot]);
            }
        }
        if (prev >= 0 && !correct_and_store(prev, prev_sig, it - 1, B0 + prv_buf * kL * P, Sprev)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int j = 0; j < S; ++j) Sprev[j] = Sl[j];
        prev = tile;
        prev_sig = sig;
        if (next < 0) break;
        tile = next;
        sig = next_sig;
        cur_buf = nxt_buf;
        ++it;
    }
    if (ok) correct_and_store(prev, prev_sig, it, B0 + cur_buf * kL * P, Sprev);
    cp_async_wait_all();
}

// The body of one class as a function of its own (not inlined): the single batch kernel calls it
// per class, so that the register allocator treats each class's body apart (inlining all 32 into
// one function costs spills and three times the build time).
template <int K, bool NORM, int N>
__device__ __noinline__ void batch_entry(BatchParams<K> p, float4 *smem4) {
    batch_body<K, NORM, N>(p, smem4);
}

template <int K, int N>
constexpr size_t batch_smem_bytes() {
    using Dm = LaneDims<K, N, kBatchW>;
    return sizeof(float) * (static_cast<size_t>(kBatchW) * 3 * kL * (N + 4) + kBatchW * kL * Dm::RSP +
                            4 * kBatchW * Dm::S + 2 * Dm::S + 2 * kBatchW * ((Dm::S + 3) / 4) * 4);
}

}  // namespace sosk
