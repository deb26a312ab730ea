// Instantiations of the single-signal DC-CR kernel for N = 32 (one translation unit
// each, so that the build compiles them in parallel).
#include "sosfilt_dccr.cuh"

namespace sosk {

template <int K, bool NORM, int LBM>
cudaError_t launch_one_32(const PassParams &p, long long grid, cudaStream_t s) {
    constexpr int N = 32;
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

template cudaError_t launch_one_32<1, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<1, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<2, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<2, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<3, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<3, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<4, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<4, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<5, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<5, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<6, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<6, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<7, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<7, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<8, false, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<8, true, 4>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<8, true, 1>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<8, true, 2>(const PassParams &, long long, cudaStream_t);
template cudaError_t launch_one_32<8, true, 8>(const PassParams &, long long, cudaStream_t);

}  // namespace sosk
