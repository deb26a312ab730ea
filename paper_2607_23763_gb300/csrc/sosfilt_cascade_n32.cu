// Instantiations of the persistent cascade-carry kernel for N = 32 (one translation unit
// per N, so that the build compiles them in parallel).
#include "sosfilt_cascade.cuh"

namespace sosk {

namespace {
constexpr int kW32 = 8;

template <int K>
size_t smem_bytes_32() {
    using Dm = CasDims<K>;
    return sizeof(float) * (static_cast<size_t>(2) * kW32 * kL * (32 + 4) + Dm::TAB + 2 * Dm::S + 4 * kW32 * Dm::S + Dm::S);
}

template <int K, bool NORM>
KernelOnce g_once;

template <int K, bool NORM>
cudaError_t launch_k_32(const CasParams<K, 32> &p, long long grid, cudaStream_t s) {
    auto kern = sos_cascade_kernel<K, 32, NORM, kW32>;
    const size_t smem = smem_bytes_32<K>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (kW32 + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_k_32() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_cascade_kernel<K, 32, NORM, kW32>, (kW32 + 1) * 32, smem_bytes_32<K>());
}
}  // namespace

template <>
cudaError_t launch_cascade<1, 32>(bool norm, const CasParams<1, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<1, true>(p, grid, s) : launch_k_32<1, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<2, 32>(bool norm, const CasParams<2, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<2, true>(p, grid, s) : launch_k_32<2, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<3, 32>(bool norm, const CasParams<3, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<3, true>(p, grid, s) : launch_k_32<3, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<4, 32>(bool norm, const CasParams<4, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<4, true>(p, grid, s) : launch_k_32<4, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<5, 32>(bool norm, const CasParams<5, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<5, true>(p, grid, s) : launch_k_32<5, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<6, 32>(bool norm, const CasParams<6, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<6, true>(p, grid, s) : launch_k_32<6, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<7, 32>(bool norm, const CasParams<7, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<7, true>(p, grid, s) : launch_k_32<7, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<8, 32>(bool norm, const CasParams<8, 32> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_32<8, true>(p, grid, s) : launch_k_32<8, false>(p, grid, s);
}

int cascade_blocks_per_sm_32(int K, bool norm) {
    switch (K) {
        case 1: return norm ? blocks_k_32<1, true>() : blocks_k_32<1, false>();
        case 2: return norm ? blocks_k_32<2, true>() : blocks_k_32<2, false>();
        case 3: return norm ? blocks_k_32<3, true>() : blocks_k_32<3, false>();
        case 4: return norm ? blocks_k_32<4, true>() : blocks_k_32<4, false>();
        case 5: return norm ? blocks_k_32<5, true>() : blocks_k_32<5, false>();
        case 6: return norm ? blocks_k_32<6, true>() : blocks_k_32<6, false>();
        case 7: return norm ? blocks_k_32<7, true>() : blocks_k_32<7, false>();
        case 8: return norm ? blocks_k_32<8, true>() : blocks_k_32<8, false>();
        default: return 0;
    }
}

size_t cascade_smem_32(int K) {
    switch (K) {
        case 1: return smem_bytes_32<1>();
        case 2: return smem_bytes_32<2>();
        case 3: return smem_bytes_32<3>();
        case 4: return smem_bytes_32<4>();
        case 5: return smem_bytes_32<5>();
        case 6: return smem_bytes_32<6>();
        case 7: return smem_bytes_32<7>();
        case 8: return smem_bytes_32<8>();
        default: return 0;
    }
}

}  // namespace sosk
