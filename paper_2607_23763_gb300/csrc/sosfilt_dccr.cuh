// Single-kernel, register-resident cascade of second-order sections for one
// long float32 signal (Sec. IV-A..B), sm_103a.
//
// One warp = one group of C = N*32 samples; lane l owns the contiguous samples
// l*N .. l*N+N-1 (Sec. IV-A), so register m across the warp is block m of the
// stride-N permuted system of Eq. 2-3.  Per section:
//   1. divide-and-conquer first level (Sec. II-E, Eqs. 19-23): multiply both
//      sides by A(-z), folding the feed-forward B(z) in, on every sample;
//   2. one-sided cyclic reduction (Eqs. 14-17) on the odd chain (m = -1 mod 2^i)
//      and the even chain (m = -2 mod 2^i) down to the lane's terminal samples
//      N-1 and N-2, both exposed before any back substitution;
//   3. the lane's zero-state terminal state (transposed direct form II) and an
//      inclusive scan of it across the 32 lanes with the N-step transition
//      T^N (the terminal-block filtering of Eq. 18 / the scan of Eq. 12);
//   4. decoupled lookback across groups with the group transition T^C
//      (Sec. II-F Eq. 25, Sec. IV-B): publish the local carry, compose the
//      predecessors' carries warp-parallel, publish the global carry;
//   5. homogeneous correction folded into back substitution: the lane's
//      incoming state enters the first row of each level (Eq. 17) and back
//      substitution recovers every sample with the state included (Eq. 24).
// The reduction and back substitution are lane-local: the only cross-lane
// traffic per section is the 5-round scan and the lookback.
#pragma once
#include "sosfilt_dccr_core.cuh"

namespace sosk {

// Warp-parallel decoupled lookback for one section of group g (g >= 1), Sec. IV-B.
// One round reads the descriptors of 32*M predecessors with independent loads (one memory
// round trip): predecessor at distance d = 32 i + lane goes to load i of `lane`.  With j the
// distance of the nearest predecessor that has posted its global carry, the incoming state is
//     z_g = sum_{d < j} (T^C)^d t[g-1-d] + (T^C)^j G[g-1-j]        (Eq. 25 unrolled),
// composed as (T^C)^lane * sum_i (T^C)^(32 i) v_i per lane and a warp sum.  If no global carry
// lies in the window, the window moves back by 32*M with the multiplier (T^C)^(32 M).
// gp[k] = (T^C)^k for k = 0..32 and gp[kPow32 + i] = (T^C)^(32 i) for i = 0..16.
template <int M>
__device__ __forceinline__ float2 lookback_resolve(const PassParams &p, const unsigned long long *d,
                                                   long long g, int lane, const float4 *gp, float2 z0,
                                                   unsigned &rounds, unsigned &waits) {
    const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
    const float4 P = __ldg(gp + lane);
    float4 Mc = make_float4(1.f, 0.f, 0.f, 1.f);
    float2 acc = make_float2(0.f, 0.f);
    long long w = 0;
    const long long t0 = clock64();
    unsigned sleep_ns = 0;
    for (;;) {
        float vx[M], vy[M];
        int st[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const long long pred = g - 1 - w - (32 * i + lane);
            if (pred >= 0) {
                unsigned long long w0, w1;
                ld_relaxed_v2(d + 2 * pred, w0, w1);
                const unsigned g0 = static_cast<unsigned>(w0 >> 32), g1 = static_cast<unsigned>(w1 >> 32);
                st[i] = (g0 == g1 && g0 == tagG) ? 2 : ((g0 == g1 && g0 == tagL) ? 1 : 0);
                vx[i] = __uint_as_float(static_cast<unsigned>(w0));
                vy[i] = __uint_as_float(static_cast<unsigned>(w1));
            } else {
                st[i] = 2;  // the signal's initial state is the global carry of group -1
                vx[i] = (pred == -1) ? z0.x : 0.f;
                vy[i] = (pred == -1) ? z0.y : 0.f;
            }
        }
        // nearest global carry (distance j) and whether every nearer predecessor is ready
        int j = 32 * M;
        bool blocked = false;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const unsigned glob = __ballot_sync(0xffffffffu, st[i] == 2);
            const unsigned inv = __ballot_sync(0xffffffffu, st[i] == 0);
            if (j == 32 * M) {
                if (glob) {
                    const int lj = __ffs(glob) - 1;
                    const unsigned need = (lj >= 31) ? 0xffffffffu : ((2u << lj) - 1u);
                    if (inv & need) blocked = true;
                    j = 32 * i + lj;
                } else if (inv) {
                    blocked = true;
                    j = 32 * i;  // stop scanning; wait
                }
            }
        }
        ++rounds;
        if (blocked) {
            ++waits;
            const bool expired = __any_sync(0xffffffffu, (clock64() - t0) > p.spin_budget);
            if (expired) {
                if (lane == 0) atomicOr(p.status, kDevErrTimeout);
                return make_float2(0.f, 0.f);
            }
            if (sleep_ns) __nanosleep(sleep_ns);
            sleep_ns = sleep_ns ? (sleep_ns < 128 ? 2 * sleep_ns : 128) : 8;
            continue;
        }
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int i = M - 1; i >= 0; --i) {
            // Horner in (T^C)^32 would need a serial chain; the table gives each power directly
            const bool use = (32 * i + lane) <= j;
            const float ux = use ? vx[i] : 0.f, uy = use ? vy[i] : 0.f;
            if (i == 0) {
                sx += ux;
                sy += uy;
            } else {
                const float4 Q = __ldg(gp + kPow32 + i);
                sx = fmaf(Q.x, ux, fmaf(Q.y, uy, sx));
                sy = fmaf(Q.z, ux, fmaf(Q.w, uy, sy));
            }
        }
        float tx = fmaf(P.x, sx, P.y * sy);
        float ty = fmaf(P.z, sx, P.w * sy);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            tx += __shfl_xor_sync(0xffffffffu, tx, o);
            ty += __shfl_xor_sync(0xffffffffu, ty, o);
        }
        acc.x = fmaf(Mc.x, tx, fmaf(Mc.y, ty, acc.x));
        acc.y = fmaf(Mc.z, tx, fmaf(Mc.w, ty, acc.y));
        if (j < 32 * M) break;
        const float4 PM = __ldg(gp + kPow32 + M);
        Mc = make_float4(fmaf(Mc.x, PM.x, Mc.y * PM.z), fmaf(Mc.x, PM.y, Mc.y * PM.w),
                         fmaf(Mc.z, PM.x, Mc.w * PM.z), fmaf(Mc.z, PM.y, Mc.w * PM.w));
        w += 32 * M;
    }
    return acc;
}

// One thread block = WARPS consecutive groups.  Per section the groups' zero-state carries are
// combined in shared memory into the block's carry, and one leader warp runs the decoupled
// lookback over block-level descriptors with the block transition S = T^(WARPS*C); each warp
// then derives its own incoming state from the block's.  Blocks draw ascending tickets, so a
// block's predecessors are always resident or finished (Sec. IV-A).
template <int K, int N, bool NORM, int WARPS, int LBM>
__global__ void __launch_bounds__(WARPS * 32) sos_dccr_kernel(const __grid_constant__ PassParams p) {
    constexpr int PITCH = N + 4;  // row pitch in floats: 16-byte rows, conflict-free 128-bit row access
    constexpr int C = N * kL;
    extern __shared__ float4 smem4[];
    __shared__ unsigned long long s_ticket;
    __shared__ float2 s_t[2][WARPS];  // groups' zero-state carries, double-buffered by section parity
    __shared__ float2 s_z[2];         // block's incoming state
    __shared__ float4 s_lp[K][32];    // (T^N)^lane per section (lane-indexed, so in shared memory)

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const bool tracing = p.trace != nullptr;
    unsigned long long t_start = 0;
    if (tracing) t_start = global_ns();
    if (threadIdx.x == 0) s_ticket = atomicAdd(p.ticket, 1ULL) - p.ticket_base;
    for (int i = threadIdx.x; i < K * 32; i += WARPS * 32) s_lp[i / 32][i % 32] = __ldg(p.lane_pow + i);
    __syncthreads();
    const long long cta = static_cast<long long>(s_ticket);
    unsigned long long *tr = (tracing && threadIdx.x == 0 && cta < p.trace_blocks)
                                 ? p.trace + static_cast<size_t>(cta) * kTraceSlots
                                 : nullptr;
    if (tr) {
        unsigned smid;
        asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
        tr[0] = static_cast<unsigned long long>(cta) + 1;
        tr[1] = t_start;
        tr[2] = global_ns();
        tr[30] = smid;
    }
    const long long g = cta * WARPS + warp;
    const long long n_cta = (p.G + WARPS - 1) / WARPS;

    float *tile = reinterpret_cast<float *>(smem4) + warp * (kL * PITCH);
    const long long base = g * C;
    const long long avail = p.n - base;  // <= 0 for a warp past the end of the signal
    const bool tail = avail < C;

    // ---- stage in: coalesced 16-byte loads -> padded rows -> registers (Sec. IV-A, Fig. 5)
#pragma unroll
    for (int j = 0; j < N / 4; ++j) {
        const int off = 4 * (j * 32 + lane);
        float4 v;
        if (!tail && p.aligned) {
            v = __ldcs(reinterpret_cast<const float4 *>(p.x + base + off));
        } else {
            const float *src = p.x + base + off;
            v.x = (off + 0 < avail) ? __ldcs(src + 0) : 0.f;
            v.y = (off + 1 < avail) ? __ldcs(src + 1) : 0.f;
            v.z = (off + 2 < avail) ? __ldcs(src + 2) : 0.f;
            v.w = (off + 3 < avail) ? __ldcs(src + 3) : 0.f;
        }
        const int row = off / N, col = off % N;
        *reinterpret_cast<float4 *>(tile + row * PITCH + col) = v;
    }
    __syncwarp();
    float r[N];
#pragma unroll
    for (int j = 0; j < N / 4; ++j) {
        const float4 v = *reinterpret_cast<const float4 *>(tile + lane * PITCH + 4 * j);
        r[4 * j + 0] = v.x;
        r[4 * j + 1] = v.y;
        r[4 * j + 2] = v.z;
        r[4 * j + 3] = v.w;
    }
    if (NORM) {
#pragma unroll
        for (int m = 0; m < N; ++m) r[m] *= p.gain;
    }
    if (tr) tr[3] = global_ns();

    // last real sample of the signal (for the final state), only in the last group
    const bool want_zf = (p.zf != nullptr) && (g == p.G - 1);
    const int plast = static_cast<int>(avail < C ? avail - 1 : C - 1);
    const int lane_last = plast / N, m_last = plast % N;

#pragma unroll
    for (int s = 0; s < K; ++s) {
        const SecCoef &c = p.sec[s];
        const int par = s & 1;
        float xin_m = 0.f, xin_m1 = 0.f;
        if (want_zf && lane == lane_last) {
            xin_m = pick<N>(r, m_last);
            xin_m1 = pick<N>(r, m_last > 0 ? m_last - 1 : 0);
        }
        const float xs1 = r[N - 1], xs2 = r[N - 2];
        Section<N, NORM>::reduce(r, c);
        // lane zero-state terminal state (transposed direct form II)
        const float yo = r[N - 1], ye = r[N - 2];
        float t1 = fmaf(c.b1, xs1, fmaf(c.b2, xs2, -fmaf(c.a1, yo, c.a2 * ye)));
        float t2 = fmaf(c.b2, xs1, -c.a2 * yo);
        // inclusive scan across lanes: Z_l = t_l + T^N Z_{l-1}
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float u1 = __shfl_up_sync(0xffffffffu, t1, 1 << k);
            const float u2 = __shfl_up_sync(0xffffffffu, t2, 1 << k);
            if (lane >= (1 << k)) {
                t1 = fmaf(c.tn[k][0], u1, fmaf(c.tn[k][1], u2, t1));
                t2 = fmaf(c.tn[k][2], u1, fmaf(c.tn[k][3], u2, t2));
            }
        }
        float zx1 = __shfl_up_sync(0xffffffffu, t1, 1);  // exclusive: state entering this lane
        float zx2 = __shfl_up_sync(0xffffffffu, t2, 1);
        if (lane == 0) zx1 = zx2 = 0.f;
        if (lane == 31) s_t[par][warp] = make_float2(t1, t2);  // group's zero-state carry
        __syncthreads();
        if (tr && s < 8) tr[4 + 3 * s] = global_ns();

        if (warp == WARPS - 1) {
            // ---- block carry and decoupled lookback over blocks (Sec. IV-B)
            const float4 *bp = p.cta_pow + s * kGrpPowStride;  // (T^(WARPS C))^k
            float T1 = 0.f, T2 = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const float *Q = c.tc[WARPS - 1 - w];
                const float2 tw = s_t[par][w];
                T1 = fmaf(Q[0], tw.x, fmaf(Q[1], tw.y, T1));
                T2 = fmaf(Q[2], tw.x, fmaf(Q[3], tw.y, T2));
            }
            unsigned long long *d = p.desc + static_cast<size_t>(s) * static_cast<size_t>(n_cta) * 2;
            const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
            float2 z0 = make_float2(0.f, 0.f);
            if (p.zi != nullptr) z0 = make_float2(p.zi[2 * s] * c.zscale, p.zi[2 * s + 1] * c.zscale);
            float2 zc;
            unsigned rounds = 0, waits = 0;
            if (cta == 0) {
                zc = z0;
            } else {
                if (lane == 0) st_relaxed_v2(d + 2 * cta, pack_word(tagL, T1), pack_word(tagL, T2));
                zc = lookback_resolve<LBM>(p, d, cta, lane, bp, z0, rounds, waits);
            }
            if (tracing && lane == 0 && cta < p.trace_blocks && s < 8)
                p.trace[static_cast<size_t>(cta) * kTraceSlots + 6 + 3 * s] =
                    (static_cast<unsigned long long>(waits) << 32) | rounds;
            if (cta + 1 < n_cta && lane == 0) {
                const float *S = c.tc[WARPS];
                const float G1 = fmaf(S[0], zc.x, fmaf(S[1], zc.y, T1));
                const float G2 = fmaf(S[2], zc.x, fmaf(S[3], zc.y, T2));
                st_relaxed_v2(d + 2 * cta, pack_word(tagG, G1), pack_word(tagG, G2));
            }
            if (lane == 0) s_z[par] = zc;
        }
        __syncthreads();
        if (tr && s < 8) tr[5 + 3 * s] = global_ns();
        // this group's incoming state: (T^C)^w z_block + sum_{v<w} (T^C)^(w-1-v) t_v
        const float2 zc = s_z[par];
        float zg1, zg2;
        {
            // warp-uniform selection among the block's constant powers (no memory access)
            zg1 = 0.f;
            zg2 = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                if (w == warp) {
                    const float *Q = c.tc[w];
                    zg1 = fmaf(Q[0], zc.x, Q[1] * zc.y);
                    zg2 = fmaf(Q[2], zc.x, Q[3] * zc.y);
#pragma unroll
                    for (int v = 0; v < w; ++v) {
                        const float *R = c.tc[w - 1 - v];
                        const float2 tv = s_t[par][v];
                        zg1 = fmaf(R[0], tv.x, fmaf(R[1], tv.y, zg1));
                        zg2 = fmaf(R[2], tv.x, fmaf(R[3], tv.y, zg2));
                    }
                }
            }
        }
        // lane incoming state: exclusive scan + (T^N)^l z_g
        const float4 Pl = s_lp[s][lane];
        const float z1 = fmaf(Pl.x, zg1, fmaf(Pl.y, zg2, zx1));
        const float z2 = fmaf(Pl.z, zg1, fmaf(Pl.w, zg2, zx2));

        Section<N, NORM>::back_substitute(r, c, z1, z2);

        if (want_zf && lane == lane_last) {
            const float ym = pick<N>(r, m_last);
            float f1, f2;
            if (m_last > 0) {
                const float ym1 = pick<N>(r, m_last - 1);
                f1 = c.b1 * xin_m + c.b2 * xin_m1 - c.a1 * ym - c.a2 * ym1;
            } else {
                f1 = c.b1 * xin_m - c.a1 * ym + z2;
            }
            f2 = c.b2 * xin_m - c.a2 * ym;
            p.zf[2 * s] = f1 * c.zscale_inv;
            p.zf[2 * s + 1] = f2 * c.zscale_inv;
        }
    }

    // ---- stage out: registers -> padded rows -> coalesced 16-byte stores
    if (tr) tr[28] = global_ns();
    __syncwarp();
#pragma unroll
    for (int j = 0; j < N / 4; ++j)
        *reinterpret_cast<float4 *>(tile + lane * PITCH + 4 * j) =
            make_float4(r[4 * j + 0], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < N / 4; ++j) {
        const int off = 4 * (j * 32 + lane);
        const int row = off / N, col = off % N;
        const float4 v = *reinterpret_cast<const float4 *>(tile + row * PITCH + col);
        if (!tail && p.aligned) {
            __stcs(reinterpret_cast<float4 *>(p.y + base + off), v);
        } else {
            float *dst = p.y + base + off;
            if (off + 0 < avail) __stcs(dst + 0, v.x);
            if (off + 1 < avail) __stcs(dst + 1, v.y);
            if (off + 2 < avail) __stcs(dst + 2, v.z);
            if (off + 3 < avail) __stcs(dst + 3, v.w);
        }
    }
    if (tr) tr[29] = global_ns();
}

}  // namespace sosk
