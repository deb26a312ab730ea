// Persistent single-signal kernel on the tensor cores, sm_103a: PH factorization of every lane's
// block (Sec. II-C) with the particular solution and the homogeneous correction (Eq. 24) evaluated
// as matrix products by tcgen05.mma, operands staged by TMA, accumulators in tensor memory.
//
// A lane owns a row of N = 64 consecutive samples.  The particular solution of a row (zero state,
// forward substitution through the banded lower-triangular system of the cascade) equals the
// product of the row with the inverse of that band matrix, which is the lower-triangular Toeplitz
// matrix of the cascade's first 64 impulse-response taps; the row's terminal 2K-word state is the
// product with the 2K x 64 matrix G of the state responses.  So for a unit of 128 rows X
// (128 x 64):
//     [Y_p | T_end] = X [T^T | G^T]                 (128 x 80 accumulator, one MMA chain)
// and after the lane scan and the carry, with the rows' true incoming states St (128 x 2K):
//     Y = Y_p + St H^T                              (accumulated on top, H the 64 x 2K basis).
// Both products run in TF32 with each float32 operand split into a TF32 head (the tensor core reads
// the upper 19 bits) and the float32 remainder, so that A B = A B_hi + A_lo B_hi + A B_lo keeps
// float32 accuracy (the dropped A_lo B_lo term is below 2^-22 relative).  The remainder of the
// input is formed in place once the first two products have read the head.
//
// A tile is two units (256 rows, 8 groups of 32 lanes, 16384 samples); tiles come from an ascending
// ticket counter (Sec. IV-A), and the carry between tiles is the PH kernels' decoupled lookback on
// the cascade state (coordinate_tile).  Warp roles per block (one block per SM):
//   warps 0, 1  coordinators, one per carry slot (tiles alternate): lookback and the groups'
//               incoming states (on two different SM schedulers: 3 % faster at orders 8 and 16
//               than both on the first)
//   warp 12     producer: tickets, TMA loads of the units' rows (the ragged last row patched in)
//   warp 2      tensor-memory owner; lane 0 issues the units' products (particular solution and
//               terminal states) and their commits
//   warp 3      split of the staged input into its TF32 remainder
//   warps 4-11  epilogue: warpgroup u (warps 4 + 4u .. 7 + 4u) takes unit u of every tile, warp
//               q of it group 4u + q, reading accumulator lanes 32q..32q+31: terminal states,
//               lane scan, fold, true row states, the correction's products (issued by the
//               warpgroup's first thread once its rows of the state operand are written: 3-5 %
//               faster than handing them to warp 2), outputs staged for TMA stores
// Pipelines: 2 input stages, 6 accumulator slots of 80 columns (tensor memory, 512 columns), one
// state-and-output buffer per epilogue warpgroup.  Every wait is bounded by the spin budget.
#pragma once
#include <cuda.h>

#include <cstring>

#include "sosfilt_lane.cuh"

namespace sosk {

constexpr int kTcN = 64;                          // samples per lane (row)
constexpr int kTcRows = 128;                      // rows of one MMA unit (four groups)
constexpr int kTcUnits = 2;                       // units per tile
constexpr int kTcW = 4 * kTcUnits;                // groups per tile
static_assert(kTcW == kTcGroups, "tile geometry");
constexpr int kTcDS = 6;                          // accumulator slots
constexpr int kTcCols = 80;                       // accumulator columns: 64 outputs, 16 state words
constexpr int kTcTmemCols = 512;                  // tensor memory allocated (kTcDS * kTcCols rounded up)
constexpr int kTcThreads = 416;                   // 13 warps
constexpr int kTcCoord1 = 1;                      // the second coordinator warp
constexpr int kTcB1 = 2 * kTcCols * 128;          // one B1 image (two K halves of 80 rows x 128 B)
constexpr int kTcImg = 2 * kTcB1 + kTcN * 128;    // B1 head, B1 remainder, B2 (H head | H remainder)
static_assert(kTcImg == kTcImageBytes, "operand image size");
constexpr int kTcXBytes = kTcRows * kTcN * 4;     // one unit of rows (two K halves of 16 KB)
constexpr int kTcOffX = kTcImg;                   // input stages
// from this many sections on, a tile's ticket waits for its accumulator slot (measured at 2^28
// samples: order 16 +22 %; orders 8 and 2 lose 2 % and 10 %, where the loads in flight matter more)
constexpr int kTcLateTicketK = 5;

template <int K>
struct TcParams {
    CUtensorMap tmx;       // x as [rows][64] float32, box 32 x 128, 128-byte swizzle
    CUtensorMap tmy;       // y, the same
    LaneParams<K> p;       // signal, carries and tables of the PH kernels (tile = kTcW groups)
    const float4 *img;     // constant operands, the shared-memory image (kTcImg bytes)
    const float *gtail;    // [2K][64] G in float32: the final state of the last lane
    long long rows;        // full rows (n / 64)
    int tail;              // samples of the partial row (n % 64)
};

template <int K>
struct TcDims {
    using Dm = LaneDims<K, kTcN, kTcW>;
    static constexpr int S = 2 * K;
    static constexpr int XS = K <= 5 ? 3 : 2;  // input stages: three where the tables leave room
    // one buffer per epilogue warpgroup: the correction's A operand [128 rows][128 B], then the
    // unit's outputs staged for the TMA stores (two K halves of 16 KB)
    static constexpr int OFF_Y = kTcOffX + XS * kTcXBytes;
    static constexpr int OFF_TAB = OFF_Y + kTcUnits * kTcXBytes;
    // tables after the staging buffers (floats): (M_N)^lane, A_C, A_T, (A_T)^32, (A_T)^31, (A_C)^v for
    // v = 1 .. W - 1, local carries, incoming states, fold prefixes, tile carries; (A_T)^lane is read
    // through L1
    static constexpr int T_ML = 0;
    static constexpr int T_AC = T_ML + 32 * Dm::MS;
    static constexpr int T_AT = T_AC + S * S;
    static constexpr int T_AT32 = T_AT + S * S;
    static constexpr int T_AT31 = T_AT32 + S * S;
    static constexpr int T_ACP = T_AT31 + S * S;
    static constexpr int T_A = T_ACP + (kTcW - 1) * S * S;
    static constexpr int T_Z = T_A + 2 * kTcW * S;
    static constexpr int T_PREF = T_Z + 2 * kTcW * S;
    static constexpr int T_AGG = T_PREF + 2 * kTcW * S;
    static constexpr int T_END = T_AGG + 2 * S;
};

template <int K>
constexpr size_t tc_smem_bytes() {
    return 1024 + TcDims<K>::OFF_TAB + sizeof(float) * TcDims<K>::T_END;  // 1024: alignment of the base
}

// ---- tcgen05, TMA and synchronisation primitives
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ unsigned long long tc_sdesc(unsigned addr) {
    return static_cast<unsigned long long>((addr & 0x3FFFF) >> 4) | (1ULL << 16) | (64ULL << 32) | (1ULL << 46) |
           (2ULL << 61);
}

// Instruction descriptor: D float32, A and B TF32 read K-major, M = 128, N columns.
__host__ __device__ constexpr unsigned tc_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<unsigned>(n >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive accumulator columns of the warp's 32 lanes: thread t receives lane base + t.
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *smem, const CUtensorMap *tm, int x, long long y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(smem)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(static_cast<int>(y)), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, int x, long long y, const void *smem) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<unsigned long long>(tm)),
                 "r"(x), "r"(static_cast<int>(y)), "r"(smem_u32(smem))
                 : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Byte offset of float c (0..31) of row r in a 128-byte-swizzled K-major block of rows: 16-byte
// chunk j of row r sits at chunk j ^ (r mod 8).
__host__ __device__ constexpr unsigned tc_swz(int r, int c) {
    return static_cast<unsigned>(r * 128 + ((((c >> 2) ^ (r & 7)) << 4) | ((c & 3) << 2)));
}

// TF32 remainder of a float32: x minus its upper 19 bits (exact).
__device__ __forceinline__ float tf32_rem(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

template <int K>
__global__ void __launch_bounds__(kTcThreads, 1) sos_tc_kernel(const __grid_constant__ TcParams<K> P) {
    using Td = TcDims<K>;
    using Dm = typename Td::Dm;
    constexpr int S = Td::S, MS = Dm::MS, XS = Td::XS;
    const LaneParams<K> &p = P.p;
    extern __shared__ unsigned char smraw[];
    unsigned char *sm =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~static_cast<uintptr_t>(1023));
    float *tabs = reinterpret_cast<float *>(sm + Td::OFF_TAB);
    float *sML = tabs + Td::T_ML;
    float *sACd = tabs + Td::T_AC;
    float *sATd = tabs + Td::T_AT;
    float *sAT32d = tabs + Td::T_AT32;
    float *sAT31d = tabs + Td::T_AT31;
    float *sACp = tabs + Td::T_ACP;
    float *pref = tabs + Td::T_PREF;
    const CoordMats mats{sATd, sAT32d, sAT31d};
    float *a_buf = tabs + Td::T_A;
    float *z_buf = tabs + Td::T_Z;
    float *agg = tabs + Td::T_AGG;
    const float *sATl = p.tab + Dm::OFF_ATL;  // (A_T)^lane, read by the coordinator through L1

    __shared__ unsigned long long full[XS], mma_a[XS], conv[XS], xfree[XS];
    __shared__ unsigned long long dfull[kTcDS], dfree[kTcDS];
    __shared__ unsigned long long corr_done[kTcUnits], patch_bar, mma_fin;
    __shared__ unsigned long long bar_local[2], bar_zready[2];
    __shared__ long long xs_tile[XS];  // tile of the unit in each input stage, -1: no more tiles
    __shared__ long long d_tile[kTcDS];   // tile of the unit in each accumulator slot, -1: no more
    __shared__ long long coord_tile[2];
    __shared__ int fold_count[2];
    __shared__ unsigned tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = p.spin_budget;
    // phase trace (diagnostics; nothing is written without a trace buffer)
    auto trace = [&](long long tile, int slot) {
        if (p.trace && tile >= 0 && tile < p.trace_tiles)
            p.trace[static_cast<size_t>(tile) * kTraceSlots + slot] = global_ns();
    };
    {
        const float4 *src = P.img;
        float4 *dst = reinterpret_cast<float4 *>(sm);
        for (int i = tid; i < kTcImg / 16; i += kTcThreads) dst[i] = __ldg(src + i);
        for (int i = tid; i < S * S; i += kTcThreads) {
            sACd[i] = __ldg(p.tab + Dm::OFF_AC + i);
            sATd[i] = __ldg(p.tab + Dm::OFF_AT + i);
            sAT32d[i] = __ldg(p.tab + Dm::OFF_AT32 + i);
            sAT31d[i] = __ldg(p.tab + Dm::OFF_AT31 + i);
        }
        for (int i = tid; i < 32 * MS; i += kTcThreads) sML[i] = __ldg(p.tab + i);
        for (int i = tid; i < (kTcW - 1) * S * S; i += kTcThreads) sACp[i] = __ldg(p.tab + Dm::OFF_ACP + i);
    }
    if (tid == 0) {
        for (int i = 0; i < XS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&mma_a[i], 1);
            mbar_init(&conv[i], 1);
            mbar_init(&xfree[i], 1);
        }
        for (int i = 0; i < kTcDS; ++i) {
            mbar_init(&dfull[i], 2);  // the MMAs' commit and the issuing thread's arrival (slot's tile)
            mbar_init(&dfree[i], 4);
        }
        for (int u = 0; u < kTcUnits; ++u) mbar_init(&corr_done[u], 1);
        mbar_init(&patch_bar, 1);
        mbar_init(&mma_fin, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_local[i], 1);
            mbar_init(&bar_zready[i], 1);
            fold_count[i] = 0;
        }
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();  // the operand image is read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;

    if (warp == 0 || warp == kTcCoord1) {
        // ------------------------------------------------------------------ coordinators
        // one per slot: tiles alternate between them, so that the lookback of one tile waits while
        // the other coordinator resolves the next
        const unsigned slot = warp == 0 ? 0 : 1;
        for (unsigned k = 0;; ++k) {
            if (!mbar_wait(&bar_local[slot], k & 1, budget, p.status)) break;
            const long long cur = coord_tile[slot];
            if (cur < 0) break;
            unsigned long long *tr =
                (p.trace && lane == 0 && cur < p.trace_tiles) ? p.trace + static_cast<size_t>(cur) * kTraceSlots : nullptr;
            if (tr) {
                unsigned smid;
                asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
                tr[0] = static_cast<unsigned long long>(cur) + 1;
                tr[1] = global_ns();
                tr[13] = smid;
            }
            coordinate_tile<K, kTcW, MS, Dm::P2, Dm::SH>(p, lane, cur, slot, budget, sATl, mats, z_buf, agg, tr);
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_zready[slot]);
            if (tr) tr[3] = global_ns();
        }
    } else if (warp == 12) {
        // ------------------------------------------------------------------ producer
        if (lane == 0) {
            unsigned i = 0, patch_phase = 0;
            bool stop = false, gave_up = false;
            while (!stop) {
                if constexpr (K >= kTcLateTicketK) {
                    // the tile's ticket is drawn only once the accumulator slot of its first unit is
                    // free, so that tiles are numbered in the order the blocks reach them and a
                    // tile's predecessors fold close to it (a shorter wait in its lookback)
                    const long long k = static_cast<long long>(i) - kTcDS;
                    if (k >= 0 && !mbar_wait(&dfree[k % kTcDS], static_cast<unsigned>(k / kTcDS) & 1u, budget, p.status)) {
                        stop = gave_up = true;
                        break;
                    }
                }
                long long tile = static_cast<long long>(atomicAdd(p.ticket, 1ULL) - p.ticket_base);
                if (tile >= p.n_tiles) tile = -1;
                trace(tile, 16);
                for (int u = 0; u < kTcUnits && !stop; ++u) {
                    const int xs = static_cast<int>(i % XS);
                    if (i >= XS && !mbar_wait(&xfree[xs], ((i / XS) - 1) & 1, budget, p.status)) {
                        stop = gave_up = true;
                        break;
                    }
                    xs_tile[xs] = tile;
                    if (tile < 0) {
                        mbar_arrive(&full[xs]);
                        stop = true;
                        break;
                    }
                    const long long row0 = (tile * kTcUnits + u) * kTcRows;
                    unsigned char *dst = sm + kTcOffX + xs * kTcXBytes;
                    // the unit holding the partial last row: its rows arrive first (rows past the
                    // tensor's end as zeros), then the row's samples are written in
                    const bool patch = P.tail > 0 && P.rows >= row0 && P.rows < row0 + kTcRows;
                    unsigned long long *bar = patch ? &patch_bar : &full[xs];
                    mbar_expect_tx(bar, kTcXBytes);
                    tma_load_2d(dst, &P.tmx, 0, row0, bar);
                    tma_load_2d(dst + kTcXBytes / 2, &P.tmx, 32, row0, bar);
                    if (u == 0) trace(tile, 17);
                    if (patch) {
                        if (!mbar_wait(&patch_bar, patch_phase, budget, p.status)) {
                            stop = gave_up = true;
                            break;
                        }
                        patch_phase ^= 1;
                        const int r = static_cast<int>(P.rows - row0);
                        const float *src = p.x + P.rows * kTcN;
                        for (int j = 0; j < P.tail; ++j)
                            *reinterpret_cast<float *>(dst + (j >> 5) * (kTcXBytes / 2) + tc_swz(r, j & 31)) = src[j];
                        fence_proxy_async_smem();
                        mbar_arrive(&full[xs]);
                    }
                    ++i;
                }
            }
            // when a wait gave up, the loads still in flight complete before the block exits (the last
            // XS units sit in distinct stages with no arrival after theirs, so their phases are the
            // current ones); after the end of the tiles the consumers take every unit issued
            if (gave_up)
                for (unsigned k = 0; k < XS && k < i; ++k) {
                    const unsigned u = i - 1 - k;
                    mbar_wait(&full[u % XS], (u / XS) & 1, budget, p.status);
                }
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr unsigned i80 = tc_idesc(kTcCols);
            const unsigned b1h = smem_u32(sm), b1l = b1h + kTcB1;
            const unsigned xb = smem_u32(sm + kTcOffX);
            // units through the first products (ia), through the remainder (ib); the corrections are
            // issued by the epilogue warpgroups
            unsigned ia = 0, ib = 0;
            bool no_more = false, term_sent = false;
            long long t_idle = clock64();
            auto chain = [&](unsigned d, unsigned a, unsigned b, bool first) {
                // X [128 x 64] (two halves of 32 floats) against 80 rows of B (the same halves)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    tc_mma(d, tc_sdesc(a + (k >> 2) * (kTcXBytes / 2) + (k & 3) * 32),
                           tc_sdesc(b + (k >> 2) * (kTcB1 / 2) + (k & 3) * 32), i80, (first && k == 0) ? 0u : 1u);
            };
            auto slot_free = [&](unsigned i) {
                return i < kTcDS || mbar_try_wait(&dfree[i % kTcDS], ((i / kTcDS) - 1) & 1);
            };
            for (;;) {
                bool prog = false;
                if (ib < ia && mbar_try_wait(&conv[ib % XS], (ib / XS) & 1)) {
                    tc_fence_after();
                    chain(tmem + (ib % kTcDS) * kTcCols, xb + (ib % XS) * kTcXBytes, b1h, false);  // X_lo B_hi
                    tc_commit(&xfree[ib % XS]);
                    tc_commit(&dfull[ib % kTcDS]);
                    if (ib % kTcUnits == 0) trace(d_tile[ib % kTcDS], 19);
                    ++ib;
                    prog = true;
                }
                if (!no_more && mbar_try_wait(&full[ia % XS], (ia / XS) & 1)) {
                    const long long tile = xs_tile[ia % XS];
                    if (tile < 0) {
                        no_more = true;
                        prog = true;
                    } else if (slot_free(ia)) {
                        tc_fence_after();
                        const unsigned d = tmem + (ia % kTcDS) * kTcCols, a = xb + (ia % XS) * kTcXBytes;
                        chain(d, a, b1h, true);   // X B_hi
                        chain(d, a, b1l, false);  // X B_lo
                        tc_commit(&mma_a[ia % XS]);
                        if (ia % kTcUnits == 0) trace(tile, 18);
                        d_tile[ia % kTcDS] = tile;
                        mbar_arrive(&dfull[ia % kTcDS]);
                        ++ia;
                        prog = true;
                    }
                }
                if (no_more && !term_sent && ib == ia && slot_free(ia) && slot_free(ia + 1)) {
                    // the next slot of each warpgroup carries the end of the tiles
                    for (unsigned e = ia; e < ia + kTcUnits; ++e) {
                        d_tile[e % kTcDS] = -1;
                        mbar_arrive(&dfull[e % kTcDS]);
                        mbar_arrive(&dfull[e % kTcDS]);
                    }
                    term_sent = true;
                    prog = true;
                }
                if (term_sent) break;
                if (prog) {
                    t_idle = clock64();
                } else if (clock64() - t_idle > budget) {
                    atomicOr(p.status, kDevErrTimeout);
                    break;
                } else {
                    __nanosleep(32);  // leave the scheduler to the epilogue warps beside this one
                }
            }
            // every product issued has completed before tensor memory is released
            tc_commit(&mma_fin);
            mbar_wait(&mma_fin, 0, budget, p.status);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ------------------------------------------------------------------ epilogue
        const int u = (warp - 4) >> 2, q = warp & 3;  // unit of every tile, group 4u + q of the tile
        const int v = 4 * u + q;
        const int r = 32 * q + lane;  // row within the unit
        const bool lead = q == 0 && lane == 0;  // issues the warpgroup's stores
        const unsigned tl = tmem + (static_cast<unsigned>(32 * q) << 16);
        unsigned char *buf = sm + Td::OFF_Y + u * kTcXBytes;  // state operand, then the staged outputs
        const ParamSecs<K> cs{p};
        const bool want_zf = p.zf != nullptr;
        const long long g_last = p.G - 1;
        const int lane_last = static_cast<int>(((p.n - 1) - g_last * (32LL * kTcN)) / kTcN);
        float Sl[S], Sp[S];
        long long prev = -1;
        unsigned jt = 0, c = 0;
        for (;;) {
            // terminal states and lane scan of this warp's group of the next tile
            const unsigned i = jt * kTcUnits + u, ds = i % kTcDS;
            if (!mbar_wait(&dfull[ds], (i / kTcDS) & 1, budget, p.status)) break;
            const long long tile = d_tile[ds];
            const unsigned slot = jt & 1;
            const bool tw = lane == 0 && q == 0;  // this warp writes its warpgroup's trace slots
            if (tw) trace(tile, u == 0 ? 4 : 22);
            if (tile >= 0) {
                tc_fence_after();
                float tv[16];
                tc_ld16(tl + ds * kTcCols + kTcN, tv);
                float t[S];
#pragma unroll
                for (int j = 0; j < S; ++j) t[j] = tv[j];
                lane_scan<K>(cs, t, Sl, a_buf + (slot * kTcW + v) * S, lane);
                if (tw) trace(tile, u == 0 ? 7 : 23);
                // the last warp to finish folds the tile's local carries (c = a_0; c = A_C c + a_v) and
                // hands the tile to the coordinator
                __syncwarp();
                int old = 0;
                if (lane == 0) {
                    __threadfence_block();
                    old = atomicAdd(&fold_count[slot], 1);
                }
                old = __shfl_sync(0xffffffffu, old, 0);
                if (tw && u == 0) trace(tile, 8);
                if (old == kTcW - 1) {
                    __threadfence_block();
                    const float *abt = a_buf + slot * kTcW * S;
                    const int li = lane < S ? lane : 0;
                    float cc = abt[li];
#pragma unroll 1
                    for (int w = 1; w < kTcW; ++w) {
                        if (lane < S) pref[(slot * kTcW + w - 1) * S + lane] = cc;
                        cc = lane_mv<S>(sACd, cc, lane) + abt[w * S + li];
                    }
                    if (lane == 0) trace(tile, 28);
                    if (tile % kAnchor != 0 && lane < S)  // an anchor's local carry is never read
                        st_relaxed_b64(p.desc + static_cast<size_t>(tile) * 2 * S + lane,
                                       pack_word((p.epoch << 2) | 1u, cc));
                    if (lane < S) agg[slot * S + lane] = cc;
                    if (lane == 0) {
                        fold_count[slot] = 0;
                        coord_tile[slot] = tile;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar_local[slot]);
                }
            } else if (u == 0 && lead) {
                coord_tile[slot] = -1;  // this slot's coordinator stops
                mbar_arrive(&bar_local[slot]);
            }
            if (prev >= 0) {
                // correction and store of this warp's group of the previous tile, once the groups'
                // incoming states are known
                const unsigned ps = (jt - 1) & 1, pds = ((jt - 1) * kTcUnits + u) % kTcDS;
                if (tw && u == 0) trace(prev, 9);
                if (!mbar_wait(&bar_zready[ps], ((jt - 1) >> 1) & 1, budget, p.status)) break;
                if (tw && u == 0) trace(prev, 10);
                float st[S];
#pragma unroll
                for (int j = 0; j < S; ++j) st[j] = Sp[j];
                {
                    // this warp's group state Z_v = (A_C)^v Z + c_{v-1} from the tile's Z and the fold's
                    // prefix carries, into the group's row of z_buf (read back as a broadcast below)
                    const int li = lane < S ? lane : 0;
                    float *zv = z_buf + (ps * kTcW + v) * S;
                    const float z0 = z_buf[ps * kTcW * S + li];
                    const float w = v == 0 ? z0 : lane_mv<S>(sACp + (v - 1) * S * S, z0, lane) + pref[(ps * kTcW + v - 1) * S + li];
                    __syncwarp();
                    if (v > 0 && lane < S) zv[lane] = w;
                    __syncwarp();
                    lane_state_mv<K>(sML + lane * MS, zv, st);
                }
                const long long g = prev * kTcW + v;
                if (want_zf && g == g_last && lane == lane_last) {
                    // final state: the lane's zero-state state after its last sample (G restricted to
                    // the samples up to it) plus the transition of its incoming state
                    const int ml = p.m_last;
                    const float *xr = p.x + (g * 32 + lane) * kTcN;
                    float zt[S];
                    packed_mv_param<K>(p.A_tail, st, zt);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float acc = 0.f;
                        for (int j = 0; j <= ml; ++j)
                            acc = fmaf(__ldg(P.gtail + s * kTcN + (kTcN - 1 - ml) + j), xr[j], acc);
                        p.zf[s] = (acc + zt[s]) * p.sec[s >> 1].zscale_inv;
                    }
                }
                // the warpgroup's buffer is free once its last store has read it; the row's state and
                // its TF32 remainder go in as the correction's A operand
                if (lead) bulk_wait_read0();
                named_bar_sync(1 + u, 128);
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    float e[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int j = 4 * (ch & 3) + k;
                        const float sv = j < S ? st[j] : 0.f;
                        e[k] = ch < 4 ? sv : tf32_rem(sv);
                    }
                    *reinterpret_cast<float4 *>(buf + tc_swz(r, 4 * ch)) = make_float4(e[0], e[1], e[2], e[3]);
                }
                fence_proxy_async_smem();
                named_bar_sync(1 + u, 128);  // the warpgroup's rows of the operand are written
                if (tw && u == 0) trace(prev, 11);
                if (lead) {
                    // Y += St H_hi + St_lo H_hi + St H_lo: St | St_lo in the row's two 64-byte halves,
                    // H_hi | H_lo likewise; 2K <= 8 state words take one K step of 8
                    tc_fence_after();
                    const unsigned d = tmem + pds * kTcCols, sa = smem_u32(buf), b2 = smem_u32(sm) + 2 * kTcB1;
                    constexpr unsigned i64 = tc_idesc(kTcN);
#pragma unroll
                    for (int kk = 0; kk < (S > 8 ? 2 : 1); ++kk) {
                        tc_mma(d, tc_sdesc(sa + 32 * kk), tc_sdesc(b2 + 32 * kk), i64, 1u);
                        tc_mma(d, tc_sdesc(sa + 64 + 32 * kk), tc_sdesc(b2 + 32 * kk), i64, 1u);
                        tc_mma(d, tc_sdesc(sa + 32 * kk), tc_sdesc(b2 + 64 + 32 * kk), i64, 1u);
                    }
                    tc_commit(&corr_done[u]);
                    if (u == 0) trace(prev, 20);
                }
                if (!mbar_wait(&corr_done[u], c & 1, budget, p.status)) break;
                if (tw) trace(prev, u == 0 ? 12 : 24);
                ++c;
                tc_fence_after();
                float yv[kTcN];
#pragma unroll
                for (int k = 0; k < kTcN / 16; ++k) {
                    float w16[16];
                    tc_ld16(tl + pds * kTcCols + 16 * k, w16);
#pragma unroll
                    for (int j = 0; j < 16; ++j) yv[16 * k + j] = w16[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&dfree[pds]);
                // outputs: staged for two TMA stores (the correction has read the state operand; rows
                // past the end are not written); the partial last row is stored by its lane
#pragma unroll
                for (int ch = 0; ch < 16; ++ch)
                    *reinterpret_cast<float4 *>(buf + (ch >> 3) * (kTcXBytes / 2) + tc_swz(r, 4 * (ch & 7))) =
                        make_float4(yv[4 * ch], yv[4 * ch + 1], yv[4 * ch + 2], yv[4 * ch + 3]);
                const long long row0 = (prev * kTcUnits + u) * kTcRows;
                if (P.tail > 0 && row0 + r == P.rows) {
                    float *dst = p.y + P.rows * kTcN;
#pragma unroll
                    for (int j = 0; j < kTcN; ++j)
                        if (j < P.tail) dst[j] = yv[j];
                }
                fence_proxy_async_smem();
                named_bar_sync(1 + u, 128);
                if (lead && row0 < P.rows) {
                    tma_store_2d(&P.tmy, 0, row0, buf);
                    tma_store_2d(&P.tmy, 32, row0, buf + kTcXBytes / 2);
                    bulk_commit();
                }
                if (tw) trace(prev, u == 0 ? 14 : 25);
            }
            if (tile < 0) {
                // the other slot's coordinator stops too, once it has taken the previous tile (whose
                // group states were observed above), so that no phase of its barrier is skipped
                if (u == 0 && lead) {
                    coord_tile[slot ^ 1] = -1;
                    mbar_arrive(&bar_local[slot ^ 1]);
                }
                break;
            }
#pragma unroll
            for (int j = 0; j < S; ++j) Sp[j] = Sl[j];
            prev = tile;
            ++jt;
        }
        if (lead) bulk_wait0();
    } else if (warp == 3) {
        // ------------------------------------------------------------------ TF32 remainder of the input
        for (unsigned i = 0;; ++i) {
            const int xs = static_cast<int>(i % XS);
            const unsigned ph = (i / XS) & 1;
            if (!mbar_wait(&full[xs], ph, budget, p.status)) break;
            if (xs_tile[xs] < 0) break;
            if (!mbar_wait(&mma_a[xs], ph, budget, p.status)) break;
            float4 *X = reinterpret_cast<float4 *>(sm + kTcOffX + xs * kTcXBytes);
#pragma unroll 8
            for (int k = 0; k < kTcXBytes / 16 / 32; ++k) {
                const float4 v = X[lane + 32 * k];
                X[lane + 32 * k] = make_float4(tf32_rem(v.x), tf32_rem(v.y), tf32_rem(v.z), tf32_rem(v.w));
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&conv[xs]);
                if (i % kTcUnits == 0) trace(xs_tile[xs], 21);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

}  // namespace sosk
