// Instantiations of the PH-factorization kernel for five to eight sections
// (two translation units, so that the build compiles them in parallel).
#include "sosfilt_ph.cuh"

namespace sosk {

namespace {
template <int K, bool NORM>
cudaError_t launch_k(const PhParams<K> &p, long long grid, cudaStream_t s) {
    constexpr int WC = kPhWc;
    auto kern = sos_ph_kernel<K, NORM>;
    constexpr size_t smem = ph_smem_bytes<K>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (WC + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_k() {
    constexpr int WC = kPhWc;
    auto kern = sos_ph_kernel<K, NORM>;
    constexpr size_t smem = ph_smem_bytes<K>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (WC + 1) * 32, smem) != cudaSuccess) return 0;
    return nb;
}
}  // namespace

template <>
cudaError_t launch_ph<5>(bool norm, const PhParams<5> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<5, true>(p, grid, s) : launch_k<5, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<6>(bool norm, const PhParams<6> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<6, true>(p, grid, s) : launch_k<6, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<7>(bool norm, const PhParams<7> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<7, true>(p, grid, s) : launch_k<7, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<8>(bool norm, const PhParams<8> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<8, true>(p, grid, s) : launch_k<8, false>(p, grid, s);
}

int ph_blocks_per_sm_b(int K, bool norm) {
    switch (K) {
        case 5: return norm ? blocks_k<5, true>() : blocks_k<5, false>();
        case 6: return norm ? blocks_k<6, true>() : blocks_k<6, false>();
        case 7: return norm ? blocks_k<7, true>() : blocks_k<7, false>();
        case 8: return norm ? blocks_k<8, true>() : blocks_k<8, false>();
        default: return 0;
    }
}

}  // namespace sosk
