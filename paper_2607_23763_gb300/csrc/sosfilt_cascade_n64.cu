// Instantiations of the persistent cascade-carry kernel for N = 64 (one translation unit
// per N, so that the build compiles them in parallel).
#include "sosfilt_cascade.cuh"

namespace sosk {

namespace {
constexpr int kW64 = 4;

template <int K>
size_t smem_bytes_64() {
    using Dm = CasDims<K>;
    return sizeof(float) * (static_cast<size_t>(2) * kW64 * kL * (64 + 4) + Dm::TAB + 2 * Dm::S + 4 * kW64 * Dm::S + Dm::S);
}

template <int K, bool NORM>
KernelOnce g_once;

template <int K, bool NORM>
cudaError_t launch_k_64(const CasParams<K, 64> &p, long long grid, cudaStream_t s) {
    auto kern = sos_cascade_kernel<K, 64, NORM, kW64>;
    const size_t smem = smem_bytes_64<K>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (kW64 + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_k_64() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_cascade_kernel<K, 64, NORM, kW64>, (kW64 + 1) * 32, smem_bytes_64<K>());
}
}  // namespace

template <>
cudaError_t launch_cascade<1, 64>(bool norm, const CasParams<1, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<1, true>(p, grid, s) : launch_k_64<1, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<2, 64>(bool norm, const CasParams<2, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<2, true>(p, grid, s) : launch_k_64<2, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<3, 64>(bool norm, const CasParams<3, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<3, true>(p, grid, s) : launch_k_64<3, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<4, 64>(bool norm, const CasParams<4, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<4, true>(p, grid, s) : launch_k_64<4, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<5, 64>(bool norm, const CasParams<5, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<5, true>(p, grid, s) : launch_k_64<5, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<6, 64>(bool norm, const CasParams<6, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<6, true>(p, grid, s) : launch_k_64<6, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<7, 64>(bool norm, const CasParams<7, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<7, true>(p, grid, s) : launch_k_64<7, false>(p, grid, s);
}
template <>
cudaError_t launch_cascade<8, 64>(bool norm, const CasParams<8, 64> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k_64<8, true>(p, grid, s) : launch_k_64<8, false>(p, grid, s);
}

int cascade_blocks_per_sm_64(int K, bool norm) {
    switch (K) {
        case 1: return norm ? blocks_k_64<1, true>() : blocks_k_64<1, false>();
        case 2: return norm ? blocks_k_64<2, true>() : blocks_k_64<2, false>();
        case 3: return norm ? blocks_k_64<3, true>() : blocks_k_64<3, false>();
        case 4: return norm ? blocks_k_64<4, true>() : blocks_k_64<4, false>();
        case 5: return norm ? blocks_k_64<5, true>() : blocks_k_64<5, false>();
        case 6: return norm ? blocks_k_64<6, true>() : blocks_k_64<6, false>();
        case 7: return norm ? blocks_k_64<7, true>() : blocks_k_64<7, false>();
        case 8: return norm ? blocks_k_64<8, true>() : blocks_k_64<8, false>();
        default: return 0;
    }
}

size_t cascade_smem_64(int K) {
    switch (K) {
        case 1: return smem_bytes_64<1>();
        case 2: return smem_bytes_64<2>();
        case 3: return smem_bytes_64<3>();
        case 4: return smem_bytes_64<4>();
        case 5: return smem_bytes_64<5>();
        case 6: return smem_bytes_64<6>();
        case 7: return smem_bytes_64<7>();
        case 8: return smem_bytes_64<8>();
        default: return 0;
    }
}

}  // namespace sosk
