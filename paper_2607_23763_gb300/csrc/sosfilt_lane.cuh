// Persistent single-signal kernel: PH factorization of every lane's block (Sec. II-C) with lanes
// of N = 64 samples (32 as an option, two blocks per SM), a skewed particular pass in
// direct-form-I order and a column-wise correction, sm_103a.
//
// A tile is W = kLaneW consecutive groups of C = 32 N samples; compute warp w of a thread block
// filters group w of the tile, lane l the samples l N .. l N + N - 1.  Per tile:
//   1. particular solution: every lane runs its N samples through the K sections from zero state.
//      The sections run skewed: at step i section s takes sample i - s, its input being section
//      s - 1's output of step i - 1, so the K section updates of one step are independent and
//      keep the FMA pipe busy without any wait on the previous section.  Each section's poles act
//      on its numerator-filtered input, and the section then applies the next section's numerator
//      to its own output history (direct form I across the cascade): four FMAs per sample when
//      b0 = 1, with float32 rounding at the level of a sequential transposed-direct-form-II
//      cascade.  Zero state is the same in every realisation; the lane's terminal state is formed
//      in transposed direct form II from each section's last two inputs and outputs.  The samples
//      stay in the lane's row of shared memory and are overwritten in place by the particular
//      output.
//   2. lane scan (Sec. II-C's recursive doubling over the 32 lanes) on the whole cascade state,
//      section by section: M_N is block lower-triangular, so section k's words are scanned with its
//      own (T^N)^(2^r) once the lower sections' lane states are folded in through M_N's coupling
//      blocks.  Lane 31's inclusive state is the group's local carry.
//   3. a coordinator warp folds the tile's local carries, publishes the tile carry, resolves the
//      tile's incoming 2K-word state by decoupled lookback over tiles (Sec. IV-B, Eq. 25 on the
//      cascade state) and derives every group's incoming state Z.  The composition is fixed: the
//      resolved carry of the last tile at a multiple of 32 and the local carries after it, so
//      that outputs are reproducible bit for bit.
//   4. homogeneous correction (Eq. 24 once for the whole cascade): lane l's true incoming state is
//      S_l + (M_N)^l Z, and sample m of its row gains sum_j H_j(m) [S_l + (M_N)^l Z]_j.  The rows'
//      states go to shared memory and the correction runs across the rows: each lane takes V = 4
//      (N = 32: 2) consecutive samples of one row, so its V x 2K basis values H_j(m) stay in
//      registers, the loop stays small (no unrolled basis in the instruction stream) and every
//      corrected vector leaves in a fully coalesced store.
// Tile t is corrected after the particular pass and lane scan of tile t + 1, so the coordinator has
// one pass to resolve it.  Tiles come from an ascending ticket counter (Sec. IV-A).  The next
// tile's input is loaded into registers during the pass (coalesced 128-bit loads) and stashed into
// the warp's free row buffer at the start of the next iteration.
#pragma once
#include "sosfilt_cascade.cuh"

namespace sosk {

// Geometry of the PH kernel for K sections, N samples per lane and W groups (compute warps) per
// tile: W = 7 with N = 64 (one block per SM, 223 registers with the register prefetch) or N = 32 (two
// blocks per SM, 128 registers); W = 10 with N = 64 (one block of 11 warps per SM: three warps on
// most schedulers, at most 168 registers, so the correction takes two samples per lane and step and
// (A_T)^lane stays in global memory, read through L1).
template <int K, int N, int W = kLaneW>
struct LaneDims {
    static constexpr int S = 2 * K;
    static constexpr int NB = K * (K + 1) / 2;
    static constexpr int NF = 4 * NB;  // floats of one packed lower block-triangular matrix
    // per-lane stride of the packed powers: an odd number of 16-byte words (conflict-free rows)
    static constexpr int MS = ((NF / 4) & 1) ? NF : NF + 4;
    static constexpr int FULL = S * S;
    static constexpr int P2 = S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;
    static constexpr int SH = 5 - (P2 == 2 ? 1 : P2 == 4 ? 2 : P2 == 8 ? 3 : 4);
    static constexpr int LQ = N / 4;             // 128-bit loads per lane per group
    static constexpr int BPS = N == 32 ? 2 : 1;  // thread blocks per SM (N = 32: 4 warps per scheduler)
    static constexpr int MAXREG = N == 32 ? 128 : W > 7 ? 168 : 255;  // registers per thread
    static constexpr int V = (N == 32 || W > 7) ? 2 : 4;  // samples per lane and step of the correction
    static constexpr int CC = N / V;             // correction chunks per row
    static constexpr int RPS = 32 / CC;          // rows per step of the column-wise correction
    static constexpr bool ATL_SHARED = BPS == 1 && W <= 7;  // (A_T)^lane in shared memory (else from L1/L2)
    // row-state pitch: S rounded up to whole 16-byte words, an odd number of them
    static constexpr int S4 = (S + 3) / 4;
    static constexpr int RSP = 4 * ((S4 & 1) ? S4 : S4 + 1);
    // table block: (M_N)^lane [32][MS], (A_T)^lane [32][MS], A_C dense column-major, the basis
    // [S][N] (read in chunks of V samples), A_T, (A_T)^32 and (A_T)^31 dense
    static constexpr int OFF_ATL = 32 * MS;
    static constexpr int OFF_AC = 64 * MS;
    static constexpr int OFF_H = OFF_AC + FULL;
    static constexpr int OFF_AT = OFF_H + N * S;
    // (A_T)^32 and (A_T)^31 dense: an anchor's resolved carry from the previous anchor's, and its
    // incoming state
    static constexpr int OFF_AT32 = OFF_AT + FULL;
    static constexpr int OFF_AT31 = OFF_AT32 + FULL;
    static constexpr int TAB = OFF_AT31 + FULL;
    // global only: (A_C)^v dense, v = 1 .. W - 1, the transitions from a tile's incoming state to its
    // groups' (read through L1, or copied by kernels with room for them)
    static constexpr int OFF_ACP = TAB;
    static constexpr int TAB_GLOBAL = OFF_ACP + (W - 1) * FULL;
    // the shared-memory copy: (M_N)^lane, (A_T)^lane when ATL_SHARED, then A_C .. A_T
    static constexpr int SM_AC = ATL_SHARED ? OFF_AC : OFF_ATL;
    static constexpr int SM_TAB = SM_AC + (TAB - OFF_AC);
};

// Section constants as the passes read them.  ParamSecs: the kernel parameters of a single-signal
// launch (compile-time section index: constant-bank operands).  RegSecs: one signal of a batch, the
// recurrence coefficients loaded into registers once per tile and the rest read through the
// read-only cache.
template <int K>
struct ParamSecs {
    const LaneParams<K> &p;
    __device__ __forceinline__ float4 c(int s) const { return p.sec[s].c; }
    __device__ __forceinline__ float b0(int s) const { return p.sec[s].b0; }
    __device__ __forceinline__ float4 tn(int s, int r) const { return p.sec[s].tn[r]; }
    __device__ __forceinline__ float4 mx(int i) const { return p.MX[i]; }
};

template <int K, bool NORM>
struct RegSecs {
    const LaneSec *sec;
    const float4 *MX;
    float4 cc[K];
    float bb[K];
    __device__ __forceinline__ RegSecs(const LaneSec *s_, const float4 *mx_) : sec(s_), MX(mx_) {
#pragma unroll
        for (int s = 0; s < K; ++s) {
            cc[s] = __ldg(&sec[s].c);
            bb[s] = NORM ? 1.f : __ldg(&sec[s].b0);
        }
    }
    __device__ __forceinline__ float4 c(int s) const { return cc[s]; }
    __device__ __forceinline__ float b0(int s) const { return bb[s]; }
    __device__ __forceinline__ float4 tn(int s, int r) const { return __ldg(&sec[s].tn[r]); }
    __device__ __forceinline__ float4 mx(int i) const { return __ldg(MX + i); }
};

template <bool B>
struct CapTag {
    static constexpr bool value = B;
};

// Particular solution of the lane's row (N samples, in place) through all K sections from zero
// state, sections skewed by one sample each; t receives the terminal state (transposed direct form
// II).  With CAPTURE, the lane with cap_lane set writes its state after sample m_last to cap.
//
// The cascade runs in direct-form-I order: section s's poles act on F_s, its input already passed
// through its own numerator (y_s = F_s - a1 y_s[-1] - a2 y_s[-2]), and section s then applies
// section s + 1's numerator to its own output history (F_{s+1} = b0' y_s + b1' y_s[-1] +
// b2' y_s[-2]), which is what it hands on.  Per sample and section that is 4 FMAs when b0 = 1, and
// every intermediate value is a numerator-filtered signal or a section output: no internal signal
// is amplified by the poles before the zeros act, as the direct-form-II state 1/A(z) x is, so the
// float32 rounding stays at the level of a sequential transposed-direct-form-II cascade also for
// sections with poles near the unit circle.  The recurrence waits on one FMA per sample (the
// y[-2] term and F enter first).
template <int K, int N, bool NORM, bool CAPTURE, class Secs>
__device__ __forceinline__ void lane_particular(const Secs &cs, float *row, float gain, float (&t)[2 * K],
                                                int m_last, bool cap_lane, float *cap) {
    constexpr int D = K - 1;             // skew of the last section
    constexpr int R0 = (4 - (D & 3)) & 3;  // a step group's first output sits R0 samples into its block
    float y1[K], y2[K], pipe[K];  // section outputs y_s[-1], y_s[-2]; pipe[s] = F_{s+1} of the last step
#pragma unroll
    for (int s = 0; s < K; ++s) y1[s] = y2[s] = pipe[s] = 0.f;
    float x1 = 0.f, x2 = 0.f;  // the last two (gained) input samples
    float cz1[K], cz2[K];      // captured state (CAPTURE only)
#pragma unroll
    for (int s = 0; s < K; ++s) cz1[s] = cz2[s] = 0.f;
    const int m_cap = (CAPTURE && cap_lane) ? m_last : -(1 << 20);
    float carry[R0 > 0 ? R0 : 1];
#pragma unroll
    for (int r = 0; r < (R0 > 0 ? R0 : 1); ++r) carry[r] = 0.f;

    // section s at sample m with input F (section s's numerator already applied); xin1, xin2 are the
    // section's last two inputs (for the captured state); returns the section's output and leaves
    // F_{s+1} in pipe[s]
    auto section = [&](int s, float F, float xin1, float xin2, bool hit, auto cap_tag) -> float {
        constexpr bool CAP = decltype(cap_tag)::value;
        const float4 c = cs.c(s);  // b1, b2, -a1, -a2
        const float y = fmaf(c.z, y1[s], fmaf(c.w, y2[s], F));
        if constexpr (CAP) {
            // transposed direct form II state after this sample: z1 = b1 x + b2 x[-1] - a1 y - a2 y[-1],
            // z2 = b2 x - a2 y
            const float z1 = fmaf(c.x, xin1, fmaf(c.y, xin2, fmaf(c.z, y, c.w * y1[s])));
            const float z2 = fmaf(c.y, xin1, c.w * y);
            cz1[s] = hit ? z1 : cz1[s];
            cz2[s] = hit ? z2 : cz2[s];
        }
        if (s + 1 < K) {
            const float4 n = cs.c(s + 1 < K ? s + 1 : s);
            pipe[s] = fmaf(n.x, y1[s], fmaf(n.y, y2[s], NORM ? y : cs.b0(s + 1 < K ? s + 1 : s) * y));
        }
        y2[s] = y1[s];
        y1[s] = y;
        return y;
    };

    float4 xn = *reinterpret_cast<const float4 *>(row);
    // steps i0 .. i0 + 3; with CAP the lane records each section's state after sample m_cap
    auto step_group = [&](int i0, auto cap_tag) {
        const float4 xv = xn;
        if (i0 + 4 < N) xn = *reinterpret_cast<const float4 *>(row + i0 + 4);
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
        float out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            // step i0 + j: from the last section down, so that pipe[s - 1] and section s - 1's output
            // history are read before section s - 1 updates them in this step
#pragma unroll
            for (int s = K - 1; s >= 1; --s) {
                const float w = section(s, pipe[s - 1], y1[s - 1], y2[s - 1], (i0 + j - s) == m_cap, cap_tag);
                if (s == K - 1) out[j] = w;
            }
            const float gx = NORM ? xs[j] * gain : xs[j];
            const float4 c0 = cs.c(0);
            const float F0 = fmaf(c0.x, x1, fmaf(c0.y, x2, NORM ? gx : cs.b0(0) * gx));
            const float w0 = section(0, F0, gx, x1, (i0 + j) == m_cap, cap_tag);
            if (K == 1) out[j] = w0;
            x2 = x1;
            x1 = gx;
        }
        // out[j] is sample i0 + j - D; the aligned block at b = i0 - D - R0 is complete
        const int b = i0 - D - R0;
        if (b >= 0) {
            float blk[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) blk[r] = r < R0 ? carry[r] : out[r - R0];
            *reinterpret_cast<float4 *>(row + b) = make_float4(blk[0], blk[1], blk[2], blk[3]);
        }
#pragma unroll
        for (int r = 0; r < R0; ++r) carry[r] = out[4 - R0 + r];
    };
    if constexpr (!CAPTURE) {
#pragma unroll 1
        for (int i0 = 0; i0 < N; i0 += 4) step_group(i0, CapTag<false>{});
    } else {
        // only the step groups in which some section passes sample m_last record (section s at step
        // m_last + s); the bounds depend on m_last alone, the same in every lane of the warp
        const int lo = (m_last / 4) * 4;
        const int hi = min(N, ((m_last + K - 1) / 4) * 4 + 4);
        int i0 = 0;
#pragma unroll 1
        for (; i0 < lo; i0 += 4) step_group(i0, CapTag<false>{});
#pragma unroll 1
        for (; i0 < hi; i0 += 4) step_group(i0, CapTag<true>{});
#pragma unroll 1
        for (; i0 < N; i0 += 4) step_group(i0, CapTag<false>{});
    }
    // drain: steps N .. N + D - 1, in which only the sections s > step - N are still running
    if constexpr (D > 0) {
        float tail[R0 + D];
#pragma unroll
        for (int r = 0; r < R0; ++r) tail[r] = carry[r];
#pragma unroll
        for (int e = 0; e < D; ++e) {
#pragma unroll
            for (int s = K - 1; s >= e + 1; --s) {
                const float w = section(s, pipe[s - 1], y1[s - 1], y2[s - 1], (N + e - s) == m_cap, CapTag<CAPTURE>{});
                if (s == K - 1) tail[R0 + e] = w;
            }
        }
#pragma unroll
        for (int r = 0; r < (R0 + D) / 4; ++r)
            *reinterpret_cast<float4 *>(row + N - D - R0 + 4 * r) =
                make_float4(tail[4 * r], tail[4 * r + 1], tail[4 * r + 2], tail[4 * r + 3]);
    } else {
        (void)carry;
    }
    // transposed direct form II state after the lane's last sample, from the last two inputs and
    // outputs of every section
#pragma unroll
    for (int s = 0; s < K; ++s) {
        const float4 c = cs.c(s);
        const float xi1 = s == 0 ? x1 : y1[s > 0 ? s - 1 : 0], xi2 = s == 0 ? x2 : y2[s > 0 ? s - 1 : 0];
        t[2 * s] = fmaf(c.x, xi1, fmaf(c.y, xi2, fmaf(c.z, y1[s], c.w * y2[s])));
        t[2 * s + 1] = fmaf(c.y, xi1, c.w * y1[s]);
    }
    if constexpr (CAPTURE) {
        if (cap_lane) {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                cap[2 * s] = cz1[s];
                cap[2 * s + 1] = cz2[s];
            }
        }
    }
}

// Cascade lane scan: from the lanes' terminal particular states t, the lane's exclusive incoming
// state S (relative to zero group state) and, in lane 31, the group's local carry a_out.
template <int K, class Secs>
__device__ __forceinline__ void lane_scan(const Secs &cs, const float (&t)[2 * K], float (&S)[2 * K], float *a_out,
                                          int lane) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float u1 = t[2 * k], u2 = t[2 * k + 1];
#pragma unroll
        for (int j = 0; j < k; ++j) {
            const float4 b = cs.mx(k * (k - 1) / 2 + j);
            u1 = fmaf(b.x, S[2 * j], fmaf(b.y, S[2 * j + 1], u1));
            u2 = fmaf(b.z, S[2 * j], fmaf(b.w, S[2 * j + 1], u2));
        }
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const float o1 = __shfl_up_sync(0xffffffffu, u1, 1 << r);
            const float o2 = __shfl_up_sync(0xffffffffu, u2, 1 << r);
            const float4 tn = cs.tn(k, r);
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

// y += A x for a packed lower block-triangular A and x in shared memory (x read as word pairs,
// broadcast).
template <int K>
__device__ __forceinline__ void lane_state_mv(const float *__restrict__ A, const float *__restrict__ x,
                                              float (&y)[2 * K]) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float y0 = y[2 * s], y1 = y[2 * s + 1];
#pragma unroll
        for (int q = 0; q <= s; ++q) {
            const float4 B = *reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + q));
            const float2 xq = *reinterpret_cast<const float2 *>(x + 2 * q);
            y0 = fmaf(B.x, xq.x, fmaf(B.y, xq.y, y0));
            y1 = fmaf(B.z, xq.x, fmaf(B.w, xq.y, y1));
        }
        y[2 * s] = y0;
        y[2 * s + 1] = y1;
    }
}

// Dense matrices the coordinator applies (column-major S x S): A_T, (A_T)^32 and (A_T)^31.
struct CoordMats {
    const float *AT, *AT32, *AT31;
};

constexpr long long kAnchor = 32;      // tiles between anchors
constexpr long long kSuperAnchor = 4;  // anchors between super-anchors

// The skewed-pass PH kernel's composition: decoupled lookback over tiles (Sec. IV-B, Eq. 25 on
// the cascade state) for tile cur's incoming 2K-word state, its resolved carry when cur is an anchor
// (the tiles at multiples of 32), and the incoming state of each of its W groups in z_buf[slot]
// (Z_0 = Z, Z_{v+1} = A_C Z_v + a_v).  Fixed composition: the resolved carry of the last anchor before
// cur and the local carries after it, so that outputs are reproducible bit for bit; the anchors form
// a chain of one hop per 32 tiles.  (The tensor-core kernel, whose tiles are resolved with less work
// around them, takes the hierarchical composition of coordinate_tile below.)
template <int K, int W, int MS, int P2, int SH>
__device__ __forceinline__ void coordinate_tile_plain(const LaneParams<K> &p, int lane, long long cur, unsigned slot,
                                                      long long budget, const float *sATl, const float *sATd,
                                                      const float *sACd, const float *a_buf, float *z_buf,
                                                      const float *agg, unsigned long long *tr) {
    constexpr int S = 2 * K;
    const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u;
    auto zinit = [&](int i) -> float { return p.zi ? p.zi[i] * p.sec[i >> 1].zscale : 0.f; };
    const float *abuf = a_buf + slot * W * S;
    const float acc_i = agg[slot * S + (lane < S ? lane : 0)];
    float tmp[S];
    unsigned long long *dcur = p.desc + static_cast<size_t>(cur) * 2 * S + S;
    float zi_lane = 0.f;
    if (cur == 0) {
        zi_lane = zinit(lane < S ? lane : 0);
    } else {
        const long long a = ((cur - 1) / 32) * 32;
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
            __nanosleep(64);  // a short nap: the successors' lookbacks wait on this tile
        }
        // sum over the predecessors of (A_T)^k v_k: each lane applies its own power, then a
        // reduce-scatter leaves word i of the sum in lane i
        packed_mv<K>(sATl + lane * MS, v, tmp);
        const float part = reduce_scatter<S, P2, SH>(tmp, lane);
        zi_lane = __shfl_sync(0xffffffffu, part, (lane < S ? lane : 0) << SH);
    }
    if (tr) tr[2] = global_ns();
    if ((cur & 31) == 0 && cur + 1 < p.n_tiles) {
        // only anchor tiles' resolved carries are read: A_T Z + tile carry
        const float gl = lane_mv<S>(sATd, zi_lane, lane) + acc_i;
        if (lane < S) st_relaxed_b64(dcur + lane, pack_word(tagG, gl));
    }
    float *zb = z_buf + slot * W * S;
#pragma unroll 1
    for (int v = 0; v < W; ++v) {
        if (lane < S) zb[v * S + lane] = zi_lane;
        if (v + 1 < W) zi_lane = lane_mv<S>(sACd, zi_lane, lane) + abuf[v * S + (lane < S ? lane : 0)];
    }
}

// Row `lane` (< 2K) of a packed lower block-triangular matrix times a vector held by every lane;
// lanes >= 2K give 0.
template <int K>
__device__ __forceinline__ float packed_row(const float *__restrict__ A, const float (&x)[2 * K], int lane) {
    float y = 0.f;
    const int sb = lane >> 1, r = lane & 1;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        if (s == sb) {
#pragma unroll
            for (int t = 0; t <= s; ++t) {
                const float4 B = *reinterpret_cast<const float4 *>(A + 4 * (s * (s + 1) / 2 + t));
                y = fmaf(r ? B.z : B.x, x[2 * t], fmaf(r ? B.w : B.y, x[2 * t + 1], y));
            }
        }
    }
    return y;
}

// One tile's work of the coordinator warp: decoupled lookback over tiles (Sec. IV-B, Eq. 25 on the
// cascade state) for tile cur's incoming 2K-word state Z, posted in row 0 of z_buf[slot], and its
// resolved carry G when cur is an anchor.  The warp correcting group v then forms the group's own
// incoming state Z_v = (A_C)^v Z + c_{v-1}, with c_v the fold's carry of groups 0 .. v under zero
// input (pref): independent products, one per warp.
// The composition is fixed, so that outputs are reproducible bit for bit:
//   * every tile first sums the local carries L of the tiles after the anchor a below it (a multiple
//     of 32): P = sum_{k=1}^{cur-1-a} (A_T)^(k-1) L(cur - k);
//   * an anchor posts W(cur) = A_T P + carry(cur) in its local-carry slot (an anchor's local carry is
//     never read); from the super-anchor A below it (multiples of 128), i = (cur - A) / 32 <= 4,
//     G(cur) = (A_T)^32 (... ((A_T)^32 G(A) + W(A + 32)) ...) + W(cur) by Horner's rule, and
//     Z = (A_T)^31 G(cur - 32) + P;
//   * a tile between anchors forms G(a) by the same Horner steps from G(A) and the anchors' W (the
//     same bits as the anchor's own) and adds (A_T)^(cur-1-a) G(a), one packed row per lane.
// So the resolved carries form a chain of one hop per 128 tiles, every tile is one hop from the
// super-anchor below it, and what waits on a carry is a few 2K x 2K products: the local carries are
// summed before it can have arrived.  A lane whose carry has arrived keeps it and stops reading.
template <int K, int W, int MS, int P2, int SH>
__device__ __forceinline__ void coordinate_tile(const LaneParams<K> &p, int lane, long long cur, unsigned slot,
                                                long long budget, const float *sATl, const CoordMats &mats,
                                                float *z_buf, const float *agg, unsigned long long *tr) {
    constexpr int S = 2 * K;
    const unsigned tagL = (p.epoch << 2) | 1u, tagG = (p.epoch << 2) | 2u, tagW = (p.epoch << 2) | 3u;
    auto zinit = [&](int i) -> float { return p.zi ? p.zi[i] * p.sec[i >> 1].zscale : 0.f; };
    const float acc_i = agg[slot * S + (lane < S ? lane : 0)];
    const int li = lane < S ? lane : 0;
    // descriptor of a tile: two slots of 2K tagged words, [0] its local carry (posted by the fold;
    // an anchor's local part W), [1] its resolved carry (anchors only)
    auto desc = [&](long long t, int k) { return p.desc + static_cast<size_t>(t) * 2 * S + k * S; };
    auto timed_out = [&](long long t_start) {
        if (__any_sync(0xffffffffu, (clock64() - t_start) > budget)) {
            if (lane == 0) atomicOr(p.status, kDevErrTimeout);
            return true;
        }
        return false;
    };
    const bool anchor = cur % kAnchor == 0 && cur + 1 < p.n_tiles;  // its carries are read
    float zi_lane = 0.f;
    if (cur == 0) {
        zi_lane = zinit(li);
        if (anchor) {
            const float gl = lane_mv<S>(mats.AT, zi_lane, lane) + acc_i;
            if (lane < S) st_relaxed_b64(desc(0, 1) + lane, pack_word(tagG, gl));
        }
    } else {
        const long long a = ((cur - 1) / kAnchor) * kAnchor;
        const int ja = static_cast<int>(cur - 1 - a);  // lane of the anchor a
        // the local carries of tiles a + 1 .. cur - 1, lane l holding tile cur - 1 - l's
        float v[S];
        {
            const long long pred = cur - 1 - lane;
            const long long t_start = clock64();
            bool have = pred <= a;  // this lane's carry is complete (kept, not read again)
#pragma unroll
            for (int q = 0; q < S; ++q) v[q] = 0.f;
            for (;;) {
                if (!have) {
                    const unsigned long long *dp = desc(pred, 0);
                    bool ok = true;
#pragma unroll
                    for (int q = 0; q < S; q += 2) {
                        unsigned long long x0, x1;
                        ld_relaxed_v2(dp + q, x0, x1);
                        ok = ok && static_cast<unsigned>(x0 >> 32) == tagL && static_cast<unsigned>(x1 >> 32) == tagL;
                        v[q] = __uint_as_float(static_cast<unsigned>(x0));
                        v[q + 1] = __uint_as_float(static_cast<unsigned>(x1));
                    }
                    have = ok;
                }
                if (__all_sync(0xffffffffu, have) || timed_out(t_start)) break;
                __nanosleep(64);  // a short nap: the successors' lookbacks wait on this tile
            }
        }
        if (tr) tr[26] = global_ns();
        // the carries the composition starts from are read before the local sum is formed, so that
        // their latency overlaps it: word li of G(A) and of the local parts W(A + 32 j) of the anchors
        // after A -- up to cur for an anchor, up to a (whose G(a) the tile forms itself) otherwise
        float g[S], h[kSuperAnchor];
        const long long A = ((cur - 1) / (kAnchor * kSuperAnchor)) * (kAnchor * kSuperAnchor);
        const int ni = anchor ? static_cast<int>((cur - A) / kAnchor) : static_cast<int>((a - A) / kAnchor) + 1;
        auto load_h = [&]() -> bool {
            bool ok = true;
#pragma unroll
            for (int j = 0; j < kSuperAnchor; ++j) {
                h[j] = 0.f;
                if (j < ni) {
                    const unsigned long long w = ld_relaxed_b64(desc(A + kAnchor * j, j == 0 ? 1 : 0) + li);
                    ok = ok && static_cast<unsigned>(w >> 32) == (j == 0 ? tagG : tagW);
                    h[j] = __uint_as_float(static_cast<unsigned>(w));
                }
            }
            return ok;
        };
        bool ready = load_h();
        // P: each lane applies its own power (A_T)^lane, a reduce-scatter leaves word i in lane i
        float pl;
        {
            float tmp[S];
            packed_mv<K>(sATl + lane * MS, v, tmp);
            const float part = reduce_scatter<S, P2, SH>(tmp, lane);
            pl = __shfl_sync(0xffffffffu, part, li << SH);
        }
        if (!anchor) {
            const long long t_start = clock64();
            while (!__all_sync(0xffffffffu, ready) && !timed_out(t_start)) {
                __nanosleep(32);
                ready = load_h();
            }
            if (tr) tr[27] = global_ns();
            float ga = h[0];  // G(A), then the resolved carries of the anchors after it, up to G(a)
#pragma unroll
            for (int j = 1; j < kSuperAnchor; ++j)
                if (j < ni) ga = lane_mv<S>(mats.AT32, ga, lane) + h[j];
#pragma unroll
            for (int q = 0; q < S; ++q) g[q] = __shfl_sync(0xffffffffu, ga, q);  // G(a) whole in every lane
            zi_lane = pl + packed_row<K>(sATl + ja * MS, g, lane);
        } else {
            const float wl = lane_mv<S>(mats.AT, pl, lane) + acc_i;  // W(cur) = A_T P + carry(cur)
            if (lane < S) st_relaxed_b64(desc(cur, 0) + lane, pack_word(tagW, wl));
            const long long t_start = clock64();
            while (!__all_sync(0xffffffffu, ready) && !timed_out(t_start)) {
                __nanosleep(32);
                ready = load_h();
            }
            if (tr) tr[27] = global_ns();
            float gprev = h[0];  // G(A), then the resolved carries of the anchors after it
#pragma unroll
            for (int j = 1; j < kSuperAnchor; ++j)
                if (j < ni) gprev = lane_mv<S>(mats.AT32, gprev, lane) + h[j];
            const float gl = lane_mv<S>(mats.AT32, gprev, lane) + wl;
            if (lane < S) st_relaxed_b64(desc(cur, 1) + lane, pack_word(tagG, gl));
            zi_lane = lane_mv<S>(mats.AT31, gprev, lane) + pl;
        }
    }
    if (tr) tr[2] = global_ns();
    // the tile's incoming state; each group's is formed by the warp that corrects it
    if (lane < S) z_buf[slot * W * S + lane] = zi_lane;
}

template <int K, int N, bool NORM, int W>
__global__ void __maxnreg__((LaneDims<K, N, W>::MAXREG)) sos_lane_kernel(const __grid_constant__ LaneParams<K> p) {
    using Dm = LaneDims<K, N, W>;
    constexpr int S = Dm::S, MS = Dm::MS, LQ = Dm::LQ, V = Dm::V, CC = Dm::CC, RPS = Dm::RPS,
                  RSP = Dm::RSP;
    constexpr int P = N + 4;  // padded row pitch (floats): conflict-free 128-bit row access
    constexpr int C = N * kL;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);  // [W][2][32][P]: two row buffers per warp
    float *tab = rows + W * 2 * kL * P;              // shared copy of the table block (SM_TAB floats)
    float *sML = tab;                                // (M_N)^lane [32][MS]
    const float *sATl = Dm::ATL_SHARED ? tab + Dm::OFF_ATL : p.tab + Dm::OFF_ATL;  // (A_T)^lane [32][MS]
    float *sACd = tab + Dm::SM_AC;                   // A_C dense column-major
    const float *sH = tab + Dm::SM_AC + (Dm::OFF_H - Dm::OFF_AC);  // basis [S][N]
    float *rowst = tab + Dm::SM_TAB;                 // [W][32][RSP] rows' true incoming states
    float *a_buf = rowst + W * kL * RSP;             // [2][W][S] local carries
    float *z_buf = a_buf + 2 * W * S;                // [2][W][S] incoming states
    float *agg = z_buf + 2 * W * S;                  // [2][S] tile carry under zero incoming state
    float *zs_tail = agg + 2 * S;                    // [S] lane-local state after the last sample
    const float *sATd = tab + Dm::SM_AC + (Dm::OFF_AT - Dm::OFF_AC);    // A_T dense column-major
    // tiles alternate between two slots; the incoming-state barrier has one per slot, so that it
    // never runs two phases ahead of a waiter
    __shared__ unsigned long long bar_local[2], bar_zready[2], bar_ticket[8];
    __shared__ long long ring[8];
    __shared__ int fold_count[2];
    __shared__ int tickets_exhausted;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long budget = p.spin_budget;

    {
        const float4 *src = reinterpret_cast<const float4 *>(p.tab);
        float4 *dst = reinterpret_cast<float4 *>(tab);
        constexpr int HEAD = (Dm::ATL_SHARED ? Dm::OFF_AC : Dm::OFF_ATL) / 4;  // float4s copied as they are
        for (int i = threadIdx.x; i < HEAD; i += blockDim.x) dst[i] = __ldg(src + i);
        for (int i = threadIdx.x; i < (Dm::TAB - Dm::OFF_AC) / 4; i += blockDim.x)
            dst[Dm::SM_AC / 4 + i] = __ldg(src + Dm::OFF_AC / 4 + i);
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
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_local[i], 1);
            mbar_init(&bar_zready[i], 1);
            fold_count[i] = 0;
        }
        tickets_exhausted = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) mbar_init(&bar_ticket[i], 1);
        // tickets of iterations 0..2; the fold of iteration k draws that of k + 3
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ring[i] = draw_ticket();
            mbar_arrive(&bar_ticket[i]);
        }
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------------ coordinator warp
        unsigned it = 0;
        for (;;) {
            const unsigned slot = it & 1;
            if (!mbar_wait(&bar_ticket[it & 7], (it >> 3) & 1, budget, p.status)) break;
            const long long cur = ring[it & 7];
            if (cur < 0) break;
            if (!mbar_wait(&bar_local[slot], (it >> 1) & 1, budget, p.status)) break;
            unsigned long long *tr =
                (p.trace && lane == 0 && cur < p.trace_tiles) ? p.trace + static_cast<size_t>(cur) * kTraceSlots : nullptr;
            if (tr) {
                unsigned smid;
                asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
                tr[0] = static_cast<unsigned long long>(cur) + 1;
                tr[1] = global_ns();
                tr[13] = smid;
            }
            coordinate_tile_plain<K, W, MS, Dm::P2, Dm::SH>(p, lane, cur, slot, budget, sATl, sATd, sACd, a_buf, z_buf,
                                                            agg, tr);
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_zready[slot]);
            if (tr) tr[3] = global_ns();
            ++it;
        }
        return;
    }

    // ---------------------------------------------------------------------- compute warps
    const int w = warp - 1;
    float *B0 = rows + w * 2 * kL * P;  // the warp's two row buffers (B0, B0 + 32 P)
    const bool want_zf = p.zf != nullptr;
    const long long g_last = p.G - 1;
    const long long p_last = p.n - 1 - g_last * C;
    const int lane_last = static_cast<int>(p_last / N);
    const int m_last = p.m_last;

    auto wtrace = [&](long long tile, int slot) {
        if (p.trace && w == 0 && lane == 0 && tile < p.trace_tiles)
            p.trace[static_cast<size_t>(tile) * kTraceSlots + slot] = global_ns();
    };
    // the group's samples, coalesced: chunk j of the lane holds samples 4 (32 j + lane) .. + 3
    float4 xq[LQ];
    auto load_regs = [&](long long tile) {
        const long long base = (tile * W + w) * C;
        const long long avail = p.n - base;
        if (avail >= C && p.aligned) {
#pragma unroll
            for (int j = 0; j < LQ; ++j) xq[j] = __ldcs(reinterpret_cast<const float4 *>(p.x + base) + j * 32 + lane);
        } else {
#pragma unroll
            for (int j = 0; j < LQ; ++j) {
                const int off = 4 * (j * 32 + lane);
                const float *src = p.x + base + off;
                xq[j].x = (off + 0 < avail) ? __ldcs(src + 0) : 0.f;
                xq[j].y = (off + 1 < avail) ? __ldcs(src + 1) : 0.f;
                xq[j].z = (off + 2 < avail) ? __ldcs(src + 2) : 0.f;
                xq[j].w = (off + 3 < avail) ? __ldcs(src + 3) : 0.f;
            }
        }
    };

    // Correction of the tile of iteration jt, whose particular output is in buffer Y and whose
    // lanes' scan states are Sl: rows' true states to shared memory, then four samples per lane
    // across the rows, stored straight to y.
    auto correct_and_store = [&](long long tile, unsigned jt, const float *Y, const float (&Sl)[S]) -> bool {
        const unsigned slot = jt & 1;
        wtrace(tile, 9);
        if (!mbar_wait(&bar_zready[slot], (jt >> 1) & 1, budget, p.status)) return false;
        wtrace(tile, 10);
        const long long g = tile * W + w;
        float st[S];
#pragma unroll
        for (int j = 0; j < S; ++j) st[j] = Sl[j];
        lane_state_mv<K>(sML + lane * MS, z_buf + (slot * W + w) * S, st);
        if (want_zf && g == g_last && lane == lane_last) {
            // final state: lane-local state after the last sample plus the transition of the lane's
            // incoming state over the samples up to it
            float zt[S];
            packed_mv_param<K>(p.A_tail, st, zt);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const float inv = p.sec[s].zscale_inv;
                p.zf[2 * s] = (zs_tail[2 * s] + zt[2 * s]) * inv;
                p.zf[2 * s + 1] = (zs_tail[2 * s + 1] + zt[2 * s + 1]) * inv;
            }
        }
        if (g >= p.G) return true;
        float *RS = rowst + w * kL * RSP;
#pragma unroll
        for (int j = 0; j < S; j += 2)
            *reinterpret_cast<float2 *>(RS + lane * RSP + j) = make_float2(st[j], st[j + 1]);
        __syncwarp();
        wtrace(tile, 11);
        const int c = lane % CC, rsub = lane / CC;
        float h[S][V];  // the lane's basis values H_j(V c + q)
#pragma unroll
        for (int j = 0; j < S; ++j) {
            if constexpr (V == 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(sH + j * N + 4 * c);
                h[j][0] = t4.x, h[j][1] = t4.y, h[j][2] = t4.z, h[j][3] = t4.w;
            } else {
                const float2 t2 = *reinterpret_cast<const float2 *>(sH + j * N + 2 * c);
                h[j][0] = t2.x, h[j][1] = t2.y;
            }
        }
        const long long base = g * C;
        const long long avail = p.n - base;
        const bool full = avail >= C && p.aligned;
#pragma unroll 2
        for (int r0 = 0; r0 < kL; r0 += RPS) {
            const int r = r0 + rsub;
            float v[V];
            if constexpr (V == 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(Y + r * P + 4 * c);
                v[0] = t4.x, v[1] = t4.y, v[2] = t4.z, v[3] = t4.w;
            } else {
                const float2 t2 = *reinterpret_cast<const float2 *>(Y + r * P + 2 * c);
                v[0] = t2.x, v[1] = t2.y;
            }
            const float *sr = RS + r * RSP;
#pragma unroll
            for (int j = 0; j < S; j += 2) {
                const float2 z = *reinterpret_cast<const float2 *>(sr + j);
#pragma unroll
                for (int q = 0; q < V; ++q) v[q] = fmaf(h[j][q], z.x, fmaf(h[j + 1][q], z.y, v[q]));
            }
            const int off = r * N + V * c;
            if (full) {
                if constexpr (V == 4)
                    __stcs(reinterpret_cast<float4 *>(p.y + base + off), make_float4(v[0], v[1], v[2], v[3]));
                else
                    __stcs(reinterpret_cast<float2 *>(p.y + base + off), make_float2(v[0], v[1]));
            } else {
                float *dst = p.y + base + off;
#pragma unroll
                for (int q = 0; q < V; ++q)
                    if (off + q < avail) dst[q] = v[q];
            }
        }
        __syncwarp();
        wtrace(tile, 12);
        return true;
    };

    if (!mbar_wait(&bar_ticket[0], 0, budget, p.status)) return;
    long long tile = ring[0];
    if (tile < 0) return;
    load_regs(tile);
    unsigned it = 0;
    long long prev = -1;
    float Sprev[S];
#pragma unroll
    for (int j = 0; j < S; ++j) Sprev[j] = 0.f;
    bool ok = true;
    for (;;) {
        const long long g = tile * W + w;
        const unsigned slot = it & 1;
        float *X = B0 + slot * kL * P;  // this tile's rows; the other buffer holds the previous tile
        wtrace(tile, 4);
        // stash the prefetched samples as rows (lane l: samples l N .. l N + N - 1)
        wtrace(tile, 14);
#pragma unroll
        for (int j = 0; j < LQ; ++j) {
            const int off = 4 * (j * 32 + lane);
            *reinterpret_cast<float4 *>(X + (off / N) * P + (off % N)) = xq[j];
        }
        __syncwarp();
        wtrace(tile, 15);
        if (!mbar_wait(&bar_ticket[(it + 1) & 7], ((it + 1) >> 3) & 1, budget, p.status)) {
            ok = false;
            break;
        }
        const long long next = ring[(it + 1) & 7];
        wtrace(tile, 5);
        if (next >= 0) load_regs(next);

        float t[S], Sl[S];
        const ParamSecs<K> cs{p};
        if (g < p.G) {
            if (want_zf && g == g_last)
                lane_particular<K, N, NORM, true>(cs, X + lane * P, p.gain, t, m_last, lane == lane_last, zs_tail);
            else
                lane_particular<K, N, NORM, false>(cs, X + lane * P, p.gain, t, m_last, false, nullptr);
            wtrace(tile, 6);
            lane_scan<K>(cs, t, Sl, a_buf + (slot * W + w) * S, lane);
        } else {
            // a group past the signal's end (the last tile is not full): nothing to filter, and its
            // local carry, zero, enters the fold as the carry of zero input
#pragma unroll
            for (int j = 0; j < S; ++j) Sl[j] = 0.f;
            if (lane < S) a_buf[(slot * W + w) * S + lane] = 0.f;
        }
        wtrace(tile, 7);
        {
            // the last warp of the tile to finish folds the groups' local carries (c = a_0;
            // c = A_C c + a_v), posts the tile's carry and draws the ticket three tiles ahead
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
                if (tile % kAnchor != 0 && lane < S)  // an anchor's local carry is never read
                    st_relaxed_b64(p.desc + static_cast<size_t>(tile) * 2 * S + lane, pack_word((p.epoch << 2) | 1u, c));
                if (lane < S) agg[slot * S + lane] = c;
                if (lane == 0) {
                    fold_count[slot] = 0;
                    ring[(it + 3) & 7] = draw_ticket();
                    mbar_arrive(&bar_ticket[(it + 3) & 7]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_local[slot]);
            }
        }
        wtrace(tile, 8);
        if (prev >= 0 && !correct_and_store(prev, it - 1, B0 + (slot ^ 1) * kL * P, Sprev)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int j = 0; j < S; ++j) Sprev[j] = Sl[j];
        prev = tile;
        if (next < 0) break;
        tile = next;
        ++it;
    }
    if (ok) correct_and_store(prev, it, B0 + (it & 1) * kL * P, Sprev);
}

template <int K, int N, int W>
constexpr size_t lane_smem_bytes() {
    using Dm = LaneDims<K, N, W>;
    return sizeof(float) * (static_cast<size_t>(W) * 2 * kL * (N + 4) + Dm::SM_TAB + W * kL * Dm::RSP +
                            4 * W * Dm::S + 2 * Dm::S + ((Dm::S + 3) / 4) * 4);
}

}  // namespace sosk
