// Instantiations of the multi-signal persistent kernel for one to eight sections.
#include "sosfilt_batch.cuh"

namespace sosk {

namespace {
template <int K, bool NORM>
KernelOnce g_once;

// One class per launch (the prepared plans' per-class form and the reference for the single kernel).
template <int K, bool NORM>
__global__ void __launch_bounds__((kBatchW + 1) * 32, 1) sos_batch_kernel(const __grid_constant__ BatchParams<K> p) {
    extern __shared__ float4 smem4[];
    batch_body<K, NORM>(p, smem4);
}

template <int K, bool NORM>
cudaError_t launch_k(const BatchParams<K> &p, long long grid, cudaStream_t s) {
    auto kern = sos_batch_kernel<K, NORM>;
    constexpr size_t smem = batch_smem_bytes<K>();
    cudaError_t e = raise_smem_once(g_once<K, NORM>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), (kBatchW + 1) * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K, bool NORM>
int blocks_k() {
    return blocks_per_sm_once(g_once<K, NORM>, sos_batch_kernel<K, NORM>, (kBatchW + 1) * 32, batch_smem_bytes<K>());
}
}  // namespace

#define SOSK_BATCH_INST(k)                                                                          \
    template <>                                                                                     \
    cudaError_t launch_batch<k>(bool norm, const BatchParams<k> &p, long long grid, cudaStream_t s) { \
        return norm ? launch_k<k, true>(p, grid, s) : launch_k<k, false>(p, grid, s);               \
    }
SOSK_BATCH_INST(1)
SOSK_BATCH_INST(2)
SOSK_BATCH_INST(3)
SOSK_BATCH_INST(4)
SOSK_BATCH_INST(5)
SOSK_BATCH_INST(6)
SOSK_BATCH_INST(7)
SOSK_BATCH_INST(8)
#undef SOSK_BATCH_INST

int batch_blocks_per_sm(int K, bool norm) {
    switch (K) {
#define SOSK_CASE(k) \
    case k: return norm ? blocks_k<k, true>() : blocks_k<k, false>();
        SOSK_CASE(1) SOSK_CASE(2) SOSK_CASE(3) SOSK_CASE(4) SOSK_CASE(5) SOSK_CASE(6) SOSK_CASE(7) SOSK_CASE(8)
#undef SOSK_CASE
        default: return 0;
    }
}

}  // namespace sosk
