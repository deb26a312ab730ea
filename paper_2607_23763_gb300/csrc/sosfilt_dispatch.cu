// Dispatch from (sections, N, normalization, lookback width) to the instantiated kernels.
#include "sosfilt_internal.h"

namespace sosk {

template <int K, bool NORM, int LBM>
cudaError_t launch_one_32(const PassParams &p, long long grid, cudaStream_t s);
template <int K, bool NORM, int LBM>
cudaError_t launch_one_64(const PassParams &p, long long grid, cudaStream_t s);
template <int K, bool NORM, int LBM>
cudaError_t launch_one_128(const PassParams &p, long long grid, cudaStream_t s);
extern template cudaError_t launch_one_32<1, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<1, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<2, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<2, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<3, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<3, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<4, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<4, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<5, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<5, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<6, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<6, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<7, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<7, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<8, false, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<8, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<8, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<8, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_32<8, true, 8>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<1, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<1, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<2, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<2, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<3, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<3, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<4, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<4, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<5, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<5, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<6, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<6, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<7, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<7, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<8, false, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<8, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<8, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<8, true, 4>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_64<8, true, 8>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<1, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<2, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<3, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<4, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<5, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<6, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<7, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<8, true, 1>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<8, true, 2>(const PassParams &, long long, cudaStream_t);
extern template cudaError_t launch_one_128<8, true, 4>(const PassParams &, long long, cudaStream_t);

int default_lbm(int N) { return N <= 32 ? 4 : N == 64 ? 2 : 1; }

bool dccr_available(int K, int N, bool norm, int lbm) {
    if (lbm == 0) lbm = default_lbm(N);
    switch (N) {
        case 32: return (K == 1 && norm == false && lbm == 4) || (K == 1 && norm == true && lbm == 4) || (K == 2 && norm == false && lbm == 4) || (K == 2 && norm == true && lbm == 4) || (K == 3 && norm == false && lbm == 4) || (K == 3 && norm == true && lbm == 4) || (K == 4 && norm == false && lbm == 4) || (K == 4 && norm == true && lbm == 4) || (K == 5 && norm == false && lbm == 4) || (K == 5 && norm == true && lbm == 4) || (K == 6 && norm == false && lbm == 4) || (K == 6 && norm == true && lbm == 4) || (K == 7 && norm == false && lbm == 4) || (K == 7 && norm == true && lbm == 4) || (K == 8 && norm == false && lbm == 4) || (K == 8 && norm == true && lbm == 1) || (K == 8 && norm == true && lbm == 2) || (K == 8 && norm == true && lbm == 4) || (K == 8 && norm == true && lbm == 8);
        case 64: return (K == 1 && norm == false && lbm == 2) || (K == 1 && norm == true && lbm == 2) || (K == 2 && norm == false && lbm == 2) || (K == 2 && norm == true && lbm == 2) || (K == 3 && norm == false && lbm == 2) || (K == 3 && norm == true && lbm == 2) || (K == 4 && norm == false && lbm == 2) || (K == 4 && norm == true && lbm == 2) || (K == 5 && norm == false && lbm == 2) || (K == 5 && norm == true && lbm == 2) || (K == 6 && norm == false && lbm == 2) || (K == 6 && norm == true && lbm == 2) || (K == 7 && norm == false && lbm == 2) || (K == 7 && norm == true && lbm == 2) || (K == 8 && norm == false && lbm == 2) || (K == 8 && norm == true && lbm == 1) || (K == 8 && norm == true && lbm == 2) || (K == 8 && norm == true && lbm == 4) || (K == 8 && norm == true && lbm == 8);
        case 128: return (K == 1 && norm == true && lbm == 1) || (K == 2 && norm == true && lbm == 1) || (K == 3 && norm == true && lbm == 1) || (K == 4 && norm == true && lbm == 1) || (K == 5 && norm == true && lbm == 1) || (K == 6 && norm == true && lbm == 1) || (K == 7 && norm == true && lbm == 1) || (K == 8 && norm == true && lbm == 1) || (K == 8 && norm == true && lbm == 2) || (K == 8 && norm == true && lbm == 4);
        default: return false;
    }
}

cudaError_t launch_dccr(int K, int N, bool norm, int lbm, const PassParams &p, long long grid, cudaStream_t s) {
    if (lbm == 0) lbm = default_lbm(N);
    if (N == 32) {
        if (K == 1 && norm == false && lbm == 4) return launch_one_32<1, false, 4>(p, grid, s);
        if (K == 1 && norm == true && lbm == 4) return launch_one_32<1, true, 4>(p, grid, s);
        if (K == 2 && norm == false && lbm == 4) return launch_one_32<2, false, 4>(p, grid, s);
        if (K == 2 && norm == true && lbm == 4) return launch_one_32<2, true, 4>(p, grid, s);
        if (K == 3 && norm == false && lbm == 4) return launch_one_32<3, false, 4>(p, grid, s);
        if (K == 3 && norm == true && lbm == 4) return launch_one_32<3, true, 4>(p, grid, s);
        if (K == 4 && norm == false && lbm == 4) return launch_one_32<4, false, 4>(p, grid, s);
        if (K == 4 && norm == true && lbm == 4) return launch_one_32<4, true, 4>(p, grid, s);
        if (K == 5 && norm == false && lbm == 4) return launch_one_32<5, false, 4>(p, grid, s);
        if (K == 5 && norm == true && lbm == 4) return launch_one_32<5, true, 4>(p, grid, s);
        if (K == 6 && norm == false && lbm == 4) return launch_one_32<6, false, 4>(p, grid, s);
        if (K == 6 && norm == true && lbm == 4) return launch_one_32<6, true, 4>(p, grid, s);
        if (K == 7 && norm == false && lbm == 4) return launch_one_32<7, false, 4>(p, grid, s);
        if (K == 7 && norm == true && lbm == 4) return launch_one_32<7, true, 4>(p, grid, s);
        if (K == 8 && norm == false && lbm == 4) return launch_one_32<8, false, 4>(p, grid, s);
        if (K == 8 && norm == true && lbm == 1) return launch_one_32<8, true, 1>(p, grid, s);
        if (K == 8 && norm == true && lbm == 2) return launch_one_32<8, true, 2>(p, grid, s);
        if (K == 8 && norm == true && lbm == 4) return launch_one_32<8, true, 4>(p, grid, s);
        if (K == 8 && norm == true && lbm == 8) return launch_one_32<8, true, 8>(p, grid, s);
    }
    if (N == 64) {
        if (K == 1 && norm == false && lbm == 2) return launch_one_64<1, false, 2>(p, grid, s);
        if (K == 1 && norm == true && lbm == 2) return launch_one_64<1, true, 2>(p, grid, s);
        if (K == 2 && norm == false && lbm == 2) return launch_one_64<2, false, 2>(p, grid, s);
        if (K == 2 && norm == true && lbm == 2) return launch_one_64<2, true, 2>(p, grid, s);
        if (K == 3 && norm == false && lbm == 2) return launch_one_64<3, false, 2>(p, grid, s);
        if (K == 3 && norm == true && lbm == 2) return launch_one_64<3, true, 2>(p, grid, s);
        if (K == 4 && norm == false && lbm == 2) return launch_one_64<4, false, 2>(p, grid, s);
        if (K == 4 && norm == true && lbm == 2) return launch_one_64<4, true, 2>(p, grid, s);
        if (K == 5 && norm == false && lbm == 2) return launch_one_64<5, false, 2>(p, grid, s);
        if (K == 5 && norm == true && lbm == 2) return launch_one_64<5, true, 2>(p, grid, s);
        if (K == 6 && norm == false && lbm == 2) return launch_one_64<6, false, 2>(p, grid, s);
        if (K == 6 && norm == true && lbm == 2) return launch_one_64<6, true, 2>(p, grid, s);
        if (K == 7 && norm == false && lbm == 2) return launch_one_64<7, false, 2>(p, grid, s);
        if (K == 7 && norm == true && lbm == 2) return launch_one_64<7, true, 2>(p, grid, s);
        if (K == 8 && norm == false && lbm == 2) return launch_one_64<8, false, 2>(p, grid, s);
        if (K == 8 && norm == true && lbm == 1) return launch_one_64<8, true, 1>(p, grid, s);
        if (K == 8 && norm == true && lbm == 2) return launch_one_64<8, true, 2>(p, grid, s);
        if (K == 8 && norm == true && lbm == 4) return launch_one_64<8, true, 4>(p, grid, s);
        if (K == 8 && norm == true && lbm == 8) return launch_one_64<8, true, 8>(p, grid, s);
    }
    if (N == 128) {
        if (K == 1 && norm == true && lbm == 1) return launch_one_128<1, true, 1>(p, grid, s);
        if (K == 2 && norm == true && lbm == 1) return launch_one_128<2, true, 1>(p, grid, s);
        if (K == 3 && norm == true && lbm == 1) return launch_one_128<3, true, 1>(p, grid, s);
        if (K == 4 && norm == true && lbm == 1) return launch_one_128<4, true, 1>(p, grid, s);
        if (K == 5 && norm == true && lbm == 1) return launch_one_128<5, true, 1>(p, grid, s);
        if (K == 6 && norm == true && lbm == 1) return launch_one_128<6, true, 1>(p, grid, s);
        if (K == 7 && norm == true && lbm == 1) return launch_one_128<7, true, 1>(p, grid, s);
        if (K == 8 && norm == true && lbm == 1) return launch_one_128<8, true, 1>(p, grid, s);
        if (K == 8 && norm == true && lbm == 2) return launch_one_128<8, true, 2>(p, grid, s);
        if (K == 8 && norm == true && lbm == 4) return launch_one_128<8, true, 4>(p, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sosk
