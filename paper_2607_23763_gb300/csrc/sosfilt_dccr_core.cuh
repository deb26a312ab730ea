// Device building blocks shared by the kernels: memory-ordering and async-copy
// primitives, and the register-resident divide-and-conquer cyclic reduction of one
// section over one group (Sec. II-E, Eqs. 14-23).
#pragma once
#include <atomic>

#include <cuda_runtime.h>

#include "sosfilt_internal.h"

namespace sosk {

// Host side of a kernel instantiation, once per device: its dynamic shared-memory limit is raised
// on the first launch (the setting lasts for the context) and its resident blocks per SM are
// queried once, so that the launch path makes no attribute or occupancy call after the first.
struct KernelOnce {
    std::atomic<unsigned long long> smem_set{0}, occ_set{0};  // one bit per device
    int occ[64] = {};
};

template <class F>
inline cudaError_t raise_smem_once(KernelOnce &k, F kern, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ULL << (dev & 63);
    if (k.smem_set.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) k.smem_set.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

template <class F>
inline int blocks_per_sm_once(KernelOnce &k, F kern, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const unsigned long long bit = 1ULL << dev;
    if (k.occ_set.load(std::memory_order_acquire) & bit) return k.occ[dev];
    if (raise_smem_once(k, kern, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) return 0;
    k.occ[dev] = nb;
    k.occ_set.fetch_or(bit, std::memory_order_acq_rel);
    return nb;
}


__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

__device__ __forceinline__ unsigned long long pack_word(unsigned tag, float v) {
    return (static_cast<unsigned long long>(tag) << 32) | __float_as_uint(v);
}

__device__ __forceinline__ void st_relaxed_v2(unsigned long long *p, unsigned long long a,
                                              unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long *p, unsigned long long &a,
                                              unsigned long long &b) {
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <int N>
__device__ __forceinline__ float pick(const float (&r)[N], int m) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) v = (j == m) ? r[j] : v;
    return v;
}

// Sample m of a lane held as (even, odd) pairs.
template <int H>
__device__ __forceinline__ float pick_pair(const float2 (&P)[H], int m) {
    // component-wise selects: a select of whole pairs is turned into a dynamically indexed (local
    // memory) array by the compiler
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        v = (m == 2 * j) ? P[j].x : v;
        v = (m == 2 * j + 1) ? P[j].y : v;
    }
    return v;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void st_relaxed_b64(unsigned long long *p, unsigned long long a) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_b64(const unsigned long long *p) {
    unsigned long long a;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(a) : "l"(p) : "memory");
    return a;
}

// mbarrier (shared::cta) primitives; waits are bounded by a cycle budget.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that may suspend the warp in hardware for up to `hint_ns` until the phase completes, so
// that a waiting warp takes no issue slots from the computing ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long *bar, unsigned parity, unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

constexpr unsigned kSuspendHintNs = 200000;  // upper bound of one hardware suspension (0.2 ms)

// Wait for the phase with the given parity to complete; false (and the timeout status bit) once
// `budget` cycles have passed.  Every retry suspends the warp (bounded by kSuspendHintNs).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long budget, int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, kSuspendHintNs)) {
        if (clock64() - t0 > budget) {
            atomicOr(status, kDevErrTimeout);
            return false;
        }
    }
    return true;
}

// Ampere-style asynchronous 16-byte global -> shared copies (L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// 16-byte copy reading the first src_bytes (0..16) bytes at gmem and zero-filling the rest; with
// src_bytes = 0 nothing is read (gmem must still be a valid 16-byte aligned address).
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
// 4-byte copy of one float (src_bytes 4) or a zero (src_bytes 0: nothing is read).
__device__ __forceinline__ void cp_async4_zfill(void *smem, const void *gmem, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bulk (TMA, non-tensor) shared -> global stores tracked by per-thread bulk groups.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_store(void *gmem, const void *smem, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem), "r"(smem_u32(smem)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int N, bool NORM>
struct Section {
    static constexpr int D = ilog2(N);

    // Steps 1-2: zero-state reduction of the lane, in place.  After it, register m
    // holds v_i[m] for the level i at which row m is eliminated (levels 1..D).
    static __device__ __forceinline__ void reduce(float (&r)[N], const SecCoef &c) {
        // first level, both parities (divide and conquer), taps of B(z) A(-z)
#pragma unroll
        for (int m = N - 1; m >= 0; --m) {
            float v = NORM ? r[m] : c.t0 * r[m];
            if (m >= 1) v = fmaf(c.t1, r[m - 1], v);
            if (m >= 2) v = fmaf(c.t2, r[m - 2], v);
            if (m >= 3) v = fmaf(c.t3, r[m - 3], v);
            if (m >= 4) v = fmaf(c.t4, r[m - 4], v);
            r[m] = v;
        }
        // levels 1 -> D on each chain (descending m keeps v_i[m - 2^(i+1)] unmodified)
#pragma unroll
        for (int i = 1; i < D; ++i) {
            const int s = 1 << i;
#pragma unroll
            for (int par = 1; par >= 0; --par) {
                const int first = par ? 2 * s - 1 : 2 * s - 2;
#pragma unroll
                for (int m = N - 2 + par; m >= first; m -= 2 * s) {
                    float v = fmaf(c.ne[i], r[m - s], r[m]);
                    if (m - 2 * s >= 0) v = fmaf(c.f[i], r[m - 2 * s], v);
                    r[m] = v;
                }
            }
        }
    }

    // Step 5: back substitution with the lane's incoming state z (scaled domain).
    static __device__ __forceinline__ void back_substitute(float (&r)[N], const SecCoef &c, float z1, float z2) {
        r[N - 1] = fmaf(c.qo[D][0], z1, fmaf(c.qo[D][1], z2, r[N - 1]));
        r[N - 2] = fmaf(c.qe[D][0], z1, fmaf(c.qe[D][1], z2, r[N - 2]));
#pragma unroll
        for (int i = D - 1; i >= 1; --i) {
            const int s = 1 << i;
#pragma unroll
            for (int par = 1; par >= 0; --par) {
                const int first = par ? s - 1 : s - 2;
#pragma unroll
                for (int m = first; m < N; m += 2 * s) {
                    float v = r[m];
                    if (m == first) {
                        v = par ? fmaf(c.qo[i][0], z1, fmaf(c.qo[i][1], z2, v))
                                : fmaf(c.qe[i][0], z1, fmaf(c.qe[i][1], z2, v));
                    }
                    if (m - s >= 0) v = fmaf(c.ne[i], r[m - s], v);
                    if (m - 2 * s >= 0) v = fmaf(c.nf[i], r[m - 2 * s], v);
                    r[m] = v;
                }
            }
        }
    }
};

// The same solve with the lane's samples held as (even, odd) pairs P[j] = (x[2j], x[2j+1]): the two
// divide-and-conquer chains run side by side in packed f32x2 FMAs (sm_100+), one instruction for
// the matching samples of both chains.  Same operations and rounding as Section.
template <int N, bool NORM>
struct SectionPair {
    static constexpr int D = ilog2(N);
    static constexpr int H = N / 2;

    static __device__ __forceinline__ void reduce(float2 (&P)[H], const SecCoef &c) {
        // first level on every sample: v1 = B(z) A(-z) x; the odd taps need the shifted pairs
        // (x[2j-1], x[2j]), built from neighbouring registers
#pragma unroll
        for (int j = H - 1; j >= 0; --j) {
            const float2 A = P[j];
            float2 v = NORM ? A : __fmul2_rn(c.p_t0, A);
            const float2 Bp = (j >= 1) ? P[j - 1] : make_float2(0.f, 0.f);
            v = __ffma2_rn(c.p_t1, make_float2(Bp.y, A.x), v);
            if (j >= 1) v = __ffma2_rn(c.p_t2, Bp, v);
            if (j >= 1) {
                const float2 Cp = (j >= 2) ? P[j - 2] : make_float2(0.f, 0.f);
                v = __ffma2_rn(c.p_t3, make_float2(Cp.y, Bp.x), v);
                if (j >= 2) v = __ffma2_rn(c.p_t4, Cp, v);
            }
            P[j] = v;
        }
        // levels i -> i+1 on both chains at once: pair j holds (m-1, m) with m = -1 mod 2^(i+1)
#pragma unroll
        for (int i = 1; i < D; ++i) {
            const int s = 1 << i;
#pragma unroll
            for (int j = H - 1; j >= s - 1; j -= s) {
                float2 v = __ffma2_rn(c.p_ne[i], P[j - s / 2], P[j]);
                if (j - s >= 0) v = __ffma2_rn(c.p_f[i], P[j - s], v);
                P[j] = v;
            }
        }
    }

    static __device__ __forceinline__ void back_substitute(float2 (&P)[H], const SecCoef &c, float z1, float z2) {
        const float2 zz1 = make_float2(z1, z1), zz2 = make_float2(z2, z2);
        P[H - 1] = __ffma2_rn(c.p_q0[D], zz1, __ffma2_rn(c.p_q1[D], zz2, P[H - 1]));
#pragma unroll
        for (int i = D - 1; i >= 1; --i) {
            const int s = 1 << i;
            const int first = s / 2 - 1;
#pragma unroll
            for (int j = first; j < H; j += s) {
                float2 v = P[j];
                if (j == first) v = __ffma2_rn(c.p_q0[i], zz1, __ffma2_rn(c.p_q1[i], zz2, v));
                if (j - s / 2 >= 0) v = __ffma2_rn(c.p_ne[i], P[j - s / 2], v);
                if (j - s >= 0) v = __ffma2_rn(c.p_nf[i], P[j - s], v);
                P[j] = v;
            }
        }
    }
};

}  // namespace sosk
