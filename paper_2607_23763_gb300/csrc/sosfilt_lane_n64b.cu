// Instantiations of the skewed-pass PH kernel for N = 64, 7 groups per tile, section counts
// 5, 6, 7, 8 (split across translation units so that the build compiles them in parallel).
#include "sosfilt_lane.cuh"

namespace sosk {

namespace {
template <int K, bool NORM>
KernelOnce g_once;

template <int K, bool NORM>
cudaError_t launch_one(const LaneParams<K> &p, long long grid, cudaStream_t s) {
    auto kern = sos_lane_kernel<K, 64, NORM, 7>;
    constexpr size_t smem = lane_smem_bytes<K, 64, 7>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (7 + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_one() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_lane_kernel<K, 64, NORM, 7>, (7 + 1) * 32,
                              lane_smem_bytes<K, 64, 7>());
}
}  // namespace

template <>
cudaError_t launch_lane<5, 64, 7>(bool norm, const LaneParams<5> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<5, true>(p, grid, s) : launch_one<5, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<6, 64, 7>(bool norm, const LaneParams<6> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<6, true>(p, grid, s) : launch_one<6, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<7, 64, 7>(bool norm, const LaneParams<7> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<7, true>(p, grid, s) : launch_one<7, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<8, 64, 7>(bool norm, const LaneParams<8> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<8, true>(p, grid, s) : launch_one<8, false>(p, grid, s);
}

int lane_blocks_per_sm_n64b(int K, bool norm) {
    switch (K) {
        case 5: return norm ? blocks_one<5, true>() : blocks_one<5, false>();
        case 6: return norm ? blocks_one<6, true>() : blocks_one<6, false>();
        case 7: return norm ? blocks_one<7, true>() : blocks_one<7, false>();
        case 8: return norm ? blocks_one<8, true>() : blocks_one<8, false>();
        default: return 0;
    }
}

}  // namespace sosk
