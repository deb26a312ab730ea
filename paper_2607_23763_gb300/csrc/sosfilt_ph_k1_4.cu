// Instantiations of the PH-factorization kernel for one to four sections
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
cudaError_t launch_ph<1>(bool norm, const PhParams<1> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<1, true>(p, grid, s) : launch_k<1, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<2>(bool norm, const PhParams<2> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<2, true>(p, grid, s) : launch_k<2, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<3>(bool norm, const PhParams<3> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<3, true>(p, grid, s) : launch_k<3, false>(p, grid, s);
}
template <>
cudaError_t launch_ph<4>(bool norm, const PhParams<4> &p, long long grid, cudaStream_t s) {
    return norm ? launch_k<4, true>(p, grid, s) : launch_k<4, false>(p, grid, s);
}

int ph_blocks_per_sm_a(int K, bool norm) {
    switch (K) {
        case 1: return norm ? blocks_k<1, true>() : blocks_k<1, false>();
        case 2: return norm ? blocks_k<2, true>() : blocks_k<2, false>();
        case 3: return norm ? blocks_k<3, true>() : blocks_k<3, false>();
        case 4: return norm ? blocks_k<4, true>() : blocks_k<4, false>();
        default: return 0;
    }
}

}  // namespace sosk
