// Instantiations of the tensor-core PH kernel (sosfilt_tc.cuh) for one to eight sections, and the
// TMA tensor maps of a launch.
#include <mutex>

#include "sosfilt_tc.cuh"

namespace sosk {

namespace {
template <int K>
KernelOnce g_once;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        cudaGetLastError();
    });
    return fn;
}

// A signal as rows of 64 float32 samples (256-byte row pitch), copied in boxes of 32 x 128 with the
// 128-byte swizzle the MMA descriptors read; rows past the end load as zeros and are not stored.
bool encode_rows(CUtensorMap *tm, const float *base, long long rows) {
    EncodeTiledFn fn = encoder();
    if (!fn || rows < 1) return false;
    const cuuint64_t dim[2] = {static_cast<cuuint64_t>(kTcN), static_cast<cuuint64_t>(rows)};
    const cuuint64_t stride[1] = {static_cast<cuuint64_t>(kTcN) * sizeof(float)};
    const cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTcRows)};
    const cuuint32_t estride[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dim, stride, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int K>
cudaError_t launch_k(const LaneParams<K> &p, const float *img, const float *gtail, long long grid, cudaStream_t s) {
    TcParams<K> P;
    std::memset(&P, 0, sizeof(P));
    P.p = p;
    P.img = reinterpret_cast<const float4 *>(img);
    P.gtail = gtail;
    P.rows = p.n / kTcN;
    P.tail = static_cast<int>(p.n % kTcN);
    if (!encode_rows(&P.tmx, p.x, P.rows) || !encode_rows(&P.tmy, p.y, P.rows)) return cudaErrorInvalidValue;
    auto kern = sos_tc_kernel<K>;
    constexpr size_t smem = tc_smem_bytes<K>();
    cudaError_t e = raise_smem_once(g_once<K>, kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), kTcThreads, smem, s>>>(P);
    return cudaGetLastError();
}

template <int K>
int blocks_k() {
    return blocks_per_sm_once(g_once<K>, sos_tc_kernel<K>, kTcThreads, tc_smem_bytes<K>());
}
}  // namespace

#define SOSK_TC_INST(k)                                                                                      \
    template <>                                                                                              \
    cudaError_t launch_tc<k>(const LaneParams<k> &p, const float *img, const float *gtail, long long grid, \
                             cudaStream_t s) {                                                               \
        return launch_k<k>(p, img, gtail, grid, s);                                                          \
    }
SOSK_TC_INST(1)
SOSK_TC_INST(2)
SOSK_TC_INST(3)
SOSK_TC_INST(4)
SOSK_TC_INST(5)
SOSK_TC_INST(6)
SOSK_TC_INST(7)
SOSK_TC_INST(8)
#undef SOSK_TC_INST

int tc_blocks_per_sm(int K) {
    switch (K) {
#define SOSK_CASE(k) \
    case k: return blocks_k<k>();
        SOSK_CASE(1) SOSK_CASE(2) SOSK_CASE(3) SOSK_CASE(4) SOSK_CASE(5) SOSK_CASE(6) SOSK_CASE(7) SOSK_CASE(8)
#undef SOSK_CASE
        default: return 0;
    }
}

}  // namespace sosk
