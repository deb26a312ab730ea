// Instantiations of the single-signal DC-CR kernel for N = 128, sections 5-8 (one translation unit
// each, so that the build compiles them in parallel).
#include "sosfilt_dccr.cuh"

namespace sosk {

template <int K, bool NORM, int LBM>
cudaError_t launch_one_128(const PassParams &p, long long grid, cudaStream_t s) {
    constexpr int N = 128;
    const size_t smem = static_cast<size_t>(kWarps) * kL * (N + 4) * sizeof(float);
    auto kern = sos_dccr_kernel<K, N, NORM, kWarps, LBM>;
    if (smem > 48 * 1024) {
        static KernelOnce once;
        cudaError_t e = raise_smem_once(once, kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<static_cast<unsigned>(grid), kWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_one_128<5, true, 1>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_128<6, true, 1>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_128<7, true, 1>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_128<8, true, 1>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_128<8, true, 2>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_128<8, true, 4>(const PassParams &, long long, cudaStream_t);

}  // namespace sosk
