// Instantiations of the double-thread-group cyclic-reduction kernel (sosfilt_dtcr.cuh) for N = 64 and
// tiles of four groups (the cyclic-reduction tables of N = 64), one to eight sections.
#include "sosfilt_dtcr.cuh"

namespace sosk {

namespace {
constexpr int kDtW = 4;

template <int K, bool NORM>
KernelOnce g_once;

template <int K, bool NORM>
cudaError_t launch_k(const CasParams<K, 64> &p, long long grid, cudaStream_t s) {
    auto kern = sos_dtcr_kernel<K, 64, NORM, kDtW>;
    constexpr size_t smem = dtcr_smem_bytes<K, 64, kDtW>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (2 * kDtW + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_k() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_dtcr_kernel<K, 64, NORM, kDtW>, (2 * kDtW + 1) * 32,
                              dtcr_smem_bytes<K, 64, kDtW>());
}
}  // namespace

#define SOSK_DTCR_INST(k)                                                                            \
    template <>                                                                                      \
    cudaError_t launch_dtcr<k>(bool norm, const CasParams<k, 64> &p, long long grid, cudaStream_t s) { \
        return norm ? launch_k<k, true>(p, grid, s) : launch_k<k, false>(p, grid, s);                \
    }
SOSK_DTCR_INST(1)
SOSK_DTCR_INST(2)
SOSK_DTCR_INST(3)
SOSK_DTCR_INST(4)
SOSK_DTCR_INST(5)
SOSK_DTCR_INST(6)
SOSK_DTCR_INST(7)
SOSK_DTCR_INST(8)
#undef SOSK_DTCR_INST

int dtcr_blocks_per_sm(int K, bool norm) {
    switch (K) {
#define SOSK_CASE(k) \
    case k: return norm ? blocks_k<k, true>() : blocks_k<k, false>();
        SOSK_CASE(1) SOSK_CASE(2) SOSK_CASE(3) SOSK_CASE(4) SOSK_CASE(5) SOSK_CASE(6) SOSK_CASE(7) SOSK_CASE(8)
#undef SOSK_CASE
        default: return 0;
    }
}

}  // namespace sosk
