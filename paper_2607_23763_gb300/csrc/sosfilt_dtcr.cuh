// Double-thread-group cyclic reduction (DTCR, Sec. IV-E): the persistent cascade-carry kernel of
// sosfilt_cascade.cuh with every group held by two warps, sm_103a.
//
// After the first divide-and-conquer level (multiplication by A(-z), Eqs. 19-23) a section's system
// splits into an even- and an odd-parity chain that are reduced and back-substituted independently
// (Eqs. 14-17).  Here the two chains of a group run on two thread groups (warps) at the same time:
// warp (g, PAR) holds, per lane, the N/2 samples of parity PAR of the lane's block, so a group has
// twice the resident warps of the single-thread-group kernel for the same staged samples.  What it
// pays is the cascade handoff: the first level of every section needs both parities of the
// section's input, and the lane's terminal state needs both parities' terminal outputs, so every
// section exchanges through shared memory with two 64-thread named barriers (one per group).
// Everything else -- tiles of W groups drawn from an ascending ticket counter, the lane scan with
// (T^N)^(2^k), the fold of the groups' local carries, the coordinator's decoupled lookback over
// tiles and the one homogeneous correction of Eq. 24 for the cascade -- is the cascade kernel's, on
// the same tables.  The output of a lane is interleaved from the two parities in shared memory and
// leaves by bulk (TMA) stores.
#pragma once
#include <type_traits>

#include "sosfilt_cascade.cuh"

namespace sosk {

// 64-thread barrier of the two warps of group g (named barrier 1 + g; 0 is __syncthreads).  Every
// lane of both warps executes it, always under conditions that are the same for the whole group.
__device__ __forceinline__ void group_bar(int g) { asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory"); }

// The same barrier, returning whether `ok` holds in every thread of the group: after a bounded wait
// that may run out in one warp and not in its partner, both warps take the same branch (a warp that
// gave up alone would leave its partner waiting at the next barrier).
__device__ __forceinline__ bool group_all(int g, bool ok) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, 64, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(ok ? 1u : 0u), "r"(1 + g)
        : "memory");
    return r != 0;
}

template <int N>
struct DtDims {
    static constexpr int H = N / 2;   // samples of one parity per lane
    static constexpr int PP = H + 4;  // parity-plane row pitch (floats): conflict-free 128-bit rows
};

// Zero-state pass of one section over the own-parity chain rr (rr[j] = sample 2j + PAR of the lane's
// block).  On entry rr is the section's input, on return its zero-state output.  own / oth: this
// warp's and the partner warp's parity plane rows of the group ([32][PP]), term: the group's
// terminal-output slots ([2][32]).  The lane's incoming state of the section comes from the lane
// scan; lane 31 of the even warp writes the group's local carry words of the section to a_out.
// tail_group: this is the signal's last group and a final state is wanted (the same in both warps);
// cap_lane: the lane holding the signal's last sample.
template <int N, bool NORM, int PAR>
__device__ __forceinline__ void dt_section(float (&rr)[N / 2], const SecCoef &c, int s, float *a_out, int lane,
                                           float *own, const float *oth, float *term, int grp, bool tail_group,
                                           bool cap_lane, int m_last, float *zs, float *tail_x) {
    using Dd = DtDims<N>;
    constexpr int H = Dd::H, D = ilog2(N);
    // publish this section's input samples of our parity; read the partner's
    float *orow = own + lane * Dd::PP;
#pragma unroll
    for (int j = 0; j < H; j += 4) *reinterpret_cast<float4 *>(orow + j) = make_float4(rr[j], rr[j + 1], rr[j + 2], rr[j + 3]);
    group_bar(grp);
    float ot[H];
    const float *prow = oth + lane * Dd::PP;
#pragma unroll
    for (int j = 0; j < H; j += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(prow + j);
        ot[j] = v.x, ot[j + 1] = v.y, ot[j + 2] = v.z, ot[j + 3] = v.w;
    }
    // the section's last two inputs: x[N-1] (odd) and x[N-2] (even)
    const float xs1 = PAR ? rr[H - 1] : ot[H - 1];
    const float xs2 = PAR ? ot[H - 1] : rr[H - 1];
    if (tail_group && cap_lane && PAR == 0) {
        // inputs at the signal's last sample and the one before it (for the final state)
        float xm = 0.f, xm1 = 0.f;
#pragma unroll
        for (int j = 0; j < H; ++j) {
            xm = (m_last == 2 * j) ? rr[j] : (m_last == 2 * j + 1) ? ot[j] : xm;
            xm1 = (m_last - 1 == 2 * j) ? rr[j] : (m_last - 1 == 2 * j + 1) ? ot[j] : xm1;
        }
        tail_x[0] = xm;
        tail_x[1] = xm1;
    }
    // first level on our parity: v[m] = (B(z) A(-z) x)[m], the five taps t0..t4 on x[m .. m-4];
    // for m = 2j + PAR, x[m - 1] and x[m - 3] are the partner's samples j - 1 + PAR and j - 2 + PAR
#pragma unroll
    for (int j = H - 1; j >= 0; --j) {
        const float x1 = (j - 1 + PAR >= 0) ? ot[j - 1 + PAR >= 0 ? j - 1 + PAR : 0] : 0.f;
        const float x2 = (j >= 1) ? rr[j >= 1 ? j - 1 : 0] : 0.f;
        const float x3 = (j - 2 + PAR >= 0) ? ot[j - 2 + PAR >= 0 ? j - 2 + PAR : 0] : 0.f;
        const float x4 = (j >= 2) ? rr[j >= 2 ? j - 2 : 0] : 0.f;
        float v = NORM ? rr[j] : c.t0 * rr[j];
        v = fmaf(c.t1, x1, v);
        v = fmaf(c.t2, x2, v);
        v = fmaf(c.t3, x3, v);
        v = fmaf(c.t4, x4, v);
        rr[j] = v;
    }
    // one-sided cyclic reduction on the chain (descending j keeps the lower rows of the level)
#pragma unroll
    for (int i = 1; i < D; ++i) {
        const int sp = 1 << i;
#pragma unroll
        for (int j = H - 1; j >= sp - 1; j -= sp) {
            float v = fmaf(c.ne[i], rr[j - sp / 2], rr[j]);
            if (j - sp >= 0) v = fmaf(c.f[i], rr[j - sp], v);
            rr[j] = v;
        }
    }
    // both terminal outputs (zero state): y[N-1] (odd) and y[N-2] (even)
    term[PAR * 32 + lane] = rr[H - 1];
    group_bar(grp);
    const float yo = PAR ? rr[H - 1] : term[32 + lane];
    const float ye = PAR ? term[lane] : rr[H - 1];
    // the lane's terminal state, scanned across the lanes with (T^N)^(2^k) (both warps alike)
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
    float z1 = __shfl_up_sync(0xffffffffu, t1, 1);
    float z2 = __shfl_up_sync(0xffffffffu, t2, 1);
    if (lane == 0) z1 = z2 = 0.f;
    if (PAR == 0 && lane == 31) {
        a_out[2 * s] = t1;
        a_out[2 * s + 1] = t2;
    }
    // back substitution on the chain with the lane's incoming state (z1, z2)
    {
        const float *q = PAR ? c.qo[D] : c.qe[D];
        rr[H - 1] = fmaf(q[0], z1, fmaf(q[1], z2, rr[H - 1]));
    }
#pragma unroll
    for (int i = D - 1; i >= 1; --i) {
        const int sp = 1 << i;
        const int first = sp / 2 - 1;
        const float *q = PAR ? c.qo[i] : c.qe[i];
#pragma unroll
        for (int j = first; j < H; j += sp) {
            float v = rr[j];
            if (j == first) v = fmaf(q[0], z1, fmaf(q[1], z2, v));
            if (j - sp / 2 >= 0) v = fmaf(c.ne[i], rr[j - sp / 2 >= 0 ? j - sp / 2 : 0], v);
            if (j - sp >= 0) v = fmaf(c.nf[i], rr[j - sp >= 0 ? j - sp : 0], v);
            rr[j] = v;
        }
    }
    if (tail_group) {
        // transposed direct form II state after the signal's last sample (zero-state part): the
        // outputs at m_last and m_last - 1 sit in different parities
        if (cap_lane) {
            float ym = 0.f, ym1 = 0.f;
#pragma unroll
            for (int j = 0; j < H; ++j) {
                ym = (m_last == 2 * j + PAR) ? rr[j] : ym;
                ym1 = (m_last - 1 == 2 * j + PAR) ? rr[j] : ym1;
            }
            // publish what this parity holds, then the even warp combines
            float *slot = tail_x + 2 + 2 * PAR;
            slot[0] = ym;
            slot[1] = ym1;
        }
        group_bar(grp);
        if (PAR == 0 && cap_lane) {
            const int pm = m_last & 1, pm1 = (m_last - 1) & 1;
            const float y_m = tail_x[2 + 2 * pm], y_m1 = tail_x[2 + 2 * pm1 + 1];
            const float xm = tail_x[0], xm1 = tail_x[1];
            float f1;
            if (m_last > 0)
                f1 = c.b1 * xm + c.b2 * xm1 - c.a1 * y_m - c.a2 * y_m1;
            else
                f1 = c.b1 * xm - c.a1 * y_m + z2;
            zs[2 * s] = f1;
            zs[2 * s + 1] = c.b2 * xm - c.a2 * y_m;
        }
        group_bar(grp);  // the slots are reused by the next section
    }
}

template <int K, int N, bool NORM, int PAR>
__device__ __forceinline__ void dt_cascade(float (&rr)[N / 2], const SecCoef *sec, float *a_out, int lane, float *own,
                                           const float *oth, float *term, int grp, bool tail_group, bool cap_lane,
                                           int m_last, float *zs, float *tail_x) {
    // the section loop stays rolled beyond two sections (instruction footprint)
    if constexpr (K <= 2) {
#pragma unroll
        for (int s = 0; s < K; ++s)
            dt_section<N, NORM, PAR>(rr, sec[s], s, a_out, lane, own, oth, term, grp, tail_group, cap_lane, m_last,
                                     zs, tail_x);
    } else {
#pragma unroll 1
        for (int s = 0; s < K; ++s)
            dt_section<N, NORM, PAR>(rr, sec[s], s, a_out, lane, own, oth, term, grp, tail_group, cap_lane, m_last,
                                     zs, tail_x);
    }
}

template <int K, int N, int W>
struct DtLayout {
    using Dm = CasDims<K>;
    using Dd = DtDims<N>;
    static constexpr int P = N + 4;                      // row pitch of the staging buffers
    static constexpr int ROWS = W * kL * P;              // one staging buffer (all groups)
    static constexpr int PLANE = kL * Dd::PP;            // one parity plane of one group
    static constexpr int OFF_X = 0;                      // [W][32][P] input of the next tile
    static constexpr int OFF_Y = ROWS;                   // [W][32][P] zero-state output, two halves per row
    static constexpr int OFF_PL = 2 * ROWS;              // [W][2][32][PP] parity planes
    static constexpr int OFF_TERM = OFF_PL + 2 * W * PLANE;  // [W][2][32] terminal outputs
    static constexpr int OFF_TAB = OFF_TERM + 2 * W * kL;   // (M_N)^lane, (A_T)^lane, A_C
    static constexpr int OFF_A = OFF_TAB + Dm::TAB;      // [2][W][S] local carries
    static constexpr int OFF_Z = OFF_A + 2 * W * Dm::S;  // [2][W][S] incoming states
    static constexpr int OFF_ZS = OFF_Z + 2 * W * Dm::S; // [S] zero-state final state
    static constexpr int OFF_AGG = OFF_ZS + Dm::S;       // [2][S] tile carries
    static constexpr int OFF_TX = OFF_AGG + 2 * Dm::S;   // [6] tail capture slots
    static constexpr int FLOATS = OFF_TX + 8;
};

template <int K, int N, bool NORM, int W>
__global__ void __maxnreg__(128)
    sos_dtcr_kernel(const __grid_constant__ CasParams<K, N> p) {
    using Dm = CasDims<K>;
    using Ly = DtLayout<K, N, W>;
    constexpr int S = Dm::S, MS = Dm::MS, H = DtDims<N>::H, PP = DtDims<N>::PP, P = Ly::P;
    constexpr int C = N * kL;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *sMl = sm + Ly::OFF_TAB;       // [32][MS]: (M_N)^lane
    float *sATl = sMl + kL * MS;         // [32][MS]: (A_T)^lane
    float *sACd = sATl + kL * MS;        // A_C dense column-major
    const float *gATd = p.tab + Dm::TAB; // A_T dense column-major (global)
    float *a_buf = sm + Ly::OFF_A;
    float *z_buf = sm + Ly::OFF_Z;
    float *zs_tail = sm + Ly::OFF_ZS;
    float *agg = sm + Ly::OFF_AGG;
    float *tail_x = sm + Ly::OFF_TX;
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

    if (warp == 0) {
        cascade_coordinator<K, N, W>(p, lane, budget, bar_local, bar_zready, bar_ticket, ring, a_buf, z_buf, agg,
                                     sATl, sACd, gATd);
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int grp = (warp - 1) >> 1;  // group of the tile
    const int par = (warp - 1) & 1;   // parity of the samples this warp holds
    float *X = sm + Ly::OFF_X + grp * kL * P;
    float *Y = sm + Ly::OFF_Y + grp * kL * P;
    float *pl = sm + Ly::OFF_PL + grp * 2 * Ly::PLANE;
    float *term = sm + Ly::OFF_TERM + grp * 2 * kL;
    const bool want_zf = p.zf != nullptr;
    const long long g_last = p.G - 1;
    const long long p_last = p.n - 1 - g_last * C;
    const int lane_last = static_cast<int>(p_last / N), m_last = static_cast<int>(p_last % N);

    // the group's input rows; the two warps issue alternate chunks (each waits for its own copies,
    // then the group barrier makes both halves visible)
    auto issue_load = [&](long long g) {
        const long long base = g * C;
        const long long avail = p.n - base;
        const float *x = p.x;
        if (avail > 0) {
            if (p.aligned) {
#pragma unroll
                for (int j = par; j < N / 4; j += 2) {
                    const int off = 4 * (j * 32 + lane);
                    const long long rem = avail - off;
                    const unsigned bytes = rem >= 4 ? 16u : rem > 0 ? static_cast<unsigned>(4 * rem) : 0u;
                    cp_async16_zfill(X + (off / N) * P + (off % N), bytes ? x + base + off : x, bytes);
                }
            } else {
#pragma unroll
                for (int j = par; j < N / 4; j += 2) {
                    const int off = 4 * (j * 32 + lane);
                    float *dst = X + (off / N) * P + (off % N);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool in = off + q < avail;
                        cp_async4_zfill(dst + q, in ? x + base + off + q : x, in ? 4u : 0u);
                    }
                }
            }
        }
        cp_async_commit();
    };

    // Correction of the tile of iteration jt from its zero-state output in Y (our parity's half of
    // each row), the interleaved row assembled in the parity planes and stored by bulk copies.
    auto correct_and_store = [&](long long tile, unsigned jt, auto par_tag) -> bool {
        constexpr int PR = decltype(par_tag)::value;
        if (!group_all(grp, mbar_wait(&bar_zready[jt & 1], (jt >> 1) & 1, budget, p.status))) return false;
        const long long g = tile * W + grp;
        const float *zb = z_buf + ((jt & 1) * W + grp) * S;
        float dz[S];
        packed_mv_sx<K>(sMl + lane * MS, zb, dz);  // the lane's incoming cascade state (M_N)^lane Z
        float *half = Y + lane * P + PR * H;
#pragma unroll
        for (int j = 0; j < H; j += 2) {
            float2 v = *reinterpret_cast<const float2 *>(half + j);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                v.x = fmaf(p.H[k][2 * j + PR], dz[k], v.x);
                v.y = fmaf(p.H[k][2 * j + 2 + PR], dz[k], v.y);
            }
            *reinterpret_cast<float2 *>(half + j) = v;
        }
        if (PR == 0 && want_zf && g == g_last && lane == lane_last) {
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
        // both halves corrected; earlier bulk stores have finished reading the planes
        bulk_wait_read0();
        group_bar(grp);
        if (g < p.G) {
            // interleave: warp PR assembles samples [PR N/2, (PR + 1) N/2) of the lane's row in its plane
            const float *ev = Y + lane * P, *od = Y + lane * P + H;
            float *dst = pl + PR * Ly::PLANE + lane * PP;
#pragma unroll
            for (int q = 0; q < H / 4; ++q) {
                const int j0 = PR * (H / 2) + 2 * q;  // samples 2 j0 .. 2 j0 + 3
                const float2 e = *reinterpret_cast<const float2 *>(ev + j0);
                const float2 o = *reinterpret_cast<const float2 *>(od + j0);
                *reinterpret_cast<float4 *>(dst + 4 * q) = make_float4(e.x, o.x, e.y, o.y);
            }
            const long long base = g * C;
            const long long avail = p.n - base;
            if (avail >= C && p.aligned) {
                fence_proxy_async_smem();
                bulk_store(p.y + base + lane * N + PR * H, dst, H * 4);
                bulk_commit();
            } else {
                const long long off0 = static_cast<long long>(lane) * N + PR * H;
#pragma unroll
                for (int q = 0; q < H; ++q)
                    if (off0 + q < avail) __stcs(p.y + base + off0 + q, dst[q]);
            }
        }
        return true;
    };

    auto body = [&](auto par_tag) {
        constexpr int PR = decltype(par_tag)::value;
        float *own = pl + PR * Ly::PLANE;
        const float *oth = pl + (1 - PR) * Ly::PLANE;
        if (!group_all(grp, mbar_wait(&bar_ticket[0], 0, budget, p.status))) return;
        long long tile = ring[0];
        if (tile < 0) return;
        issue_load(tile * W + grp);
        unsigned it = 0;
        long long prev = -1;
        bool ok = true;
        for (;;) {
            const long long g = tile * W + grp;
            cp_async_wait_all();
            group_bar(grp);
            float rr[H];
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const float4 v = *reinterpret_cast<const float4 *>(X + lane * P + 4 * j);
                rr[2 * j] = PR ? v.y : v.x;
                rr[2 * j + 1] = PR ? v.w : v.z;
            }
            if (NORM) {
#pragma unroll
                for (int j = 0; j < H; ++j) rr[j] *= p.gain;
            }
            // both warps have read X before it receives the next tile, and agree on the next ticket
            if (!group_all(grp, mbar_wait(&bar_ticket[(it + 1) & 3], ((it + 1) >> 2) & 1, budget, p.status))) {
                ok = false;
                break;
            }
            const long long next = ring[(it + 1) & 3];
            if (next >= 0) issue_load(next * W + grp);
            // the planes may still be read by the previous tile's bulk stores
            bulk_wait_read0();
            group_bar(grp);
            if (g < p.G) {
                dt_cascade<K, N, NORM, PR>(rr, p.sec, a_buf + ((it & 1) * W + grp) * S, lane, own, oth, term, grp,
                                           want_zf && g == g_last, lane == lane_last, m_last, zs_tail, tail_x);
            } else if (PR == 0 && lane < S) {
                a_buf[((it & 1) * W + grp) * S + lane] = 0.f;  // a group past the end: zero local carry
            }
            {
                // the last warp of the tile to finish folds the groups' local carries
                __syncwarp();
                int old = 0;
                if (lane == 0) {
                    __threadfence_block();
                    old = atomicAdd(&fold_count[it & 1], 1);
                }
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == 2 * W - 1) {
                    __threadfence_block();
                    const float *ab = a_buf + (it & 1) * W * S;
                    const int li = lane < S ? lane : 0;
                    float cc = ab[li];
#pragma unroll 1
                    for (int v = 1; v < W; ++v) cc = lane_mv<S>(sACd, cc, lane) + ab[v * S + li];
                    if (tile > 0 && lane < S)
                        st_relaxed_b64(p.desc + static_cast<size_t>(tile) * S + lane, pack_word((p.epoch << 2) | 1u, cc));
                    if (lane < S) agg[(it & 1) * S + lane] = cc;
                    if (lane == 0) {
                        fold_count[it & 1] = 0;
                        ring[(it + 2) & 3] = draw_ticket();
                        mbar_arrive(&bar_ticket[(it + 2) & 3]);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar_local[it & 1]);
                }
            }
            if (prev >= 0 && !correct_and_store(prev, it - 1, par_tag)) {
                ok = false;
                break;
            }
            // stash this tile's zero-state output (our half of each row) for its correction
            group_bar(grp);  // the partner has read both halves of the previous tile
#pragma unroll
            for (int j = 0; j < H; j += 4)
                *reinterpret_cast<float4 *>(Y + lane * P + PR * H + j) = make_float4(rr[j], rr[j + 1], rr[j + 2], rr[j + 3]);
            prev = tile;
            if (next < 0) break;
            tile = next;
            ++it;
        }
        if (ok) correct_and_store(prev, it, par_tag);
        bulk_wait0();
        cp_async_wait_all();
    };
    if (par == 0)
        body(std::integral_constant<int, 0>{});
    else
        body(std::integral_constant<int, 1>{});
}

template <int K, int N, int W>
constexpr size_t dtcr_smem_bytes() {
    return sizeof(float) * static_cast<size_t>(DtLayout<K, N, W>::FLOATS);
}

}  // namespace sosk
