// Instantiations of the skewed-pass PH kernel for N = 32, 7 groups per tile, section counts
// 1, 2, 3, 4 (split across translation units so that the build compiles them in parallel).
#include "sosfilt_lane.cuh"

namespace sosk {

namespace {
template <int K, bool NORM>
KernelOnce g_once;

template <int K, bool NORM>
cudaError_t launch_one(const LaneParams<K> &p, long long grid, cudaStream_t s) {
    auto kern = sos_lane_kernel<K, 32, NORM, 7>;
    constexpr size_t smem = lane_smem_bytes<K, 32, 7>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (7 + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_one() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_lane_kernel<K, 32, NORM, 7>, (7 + 1) * 32,
                              lane_smem_bytes<K, 32, 7>());
}
}  // namespace

template <>
cudaError_t launch_lane<1, 32, 7>(bool norm, const LaneParams<1> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<1, true>(p, grid, s) : launch_one<1, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<2, 32, 7>(bool norm, const LaneParams<2> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<2, true>(p, grid, s) : launch_one<2, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<3, 32, 7>(bool norm, const LaneParams<3> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<3, true>(p, grid, s) : launch_one<3, false>(p, grid, s);
}
template <>
cudaError_t launch_lane<4, 32, 7>(bool norm, const LaneParams<4> &p, long long grid, cudaStream_t s) {
    return norm ? launch_one<4, true>(p, grid, s) : launch_one<4, false>(p, grid, s);
}

int lane_blocks_per_sm_n32a(int K, bool norm) {
    switch (K) {
        case 1: return norm ? blocks_one<1, true>() : blocks_one<1, false>();
        case 2: return norm ? blocks_one<2, true>() : blocks_one<2, false>();
        case 3: return norm ? blocks_one<3, true>() : blocks_one<3, false>();
        case 4: return norm ? blocks_one<4, true>() : blocks_one<4, false>();
        default: return 0;
    }
}

}  // namespace sosk
