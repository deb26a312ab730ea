// The single persistent kernel over every class of a batch (sos_batch_all_kernel, sosfilt_batch.cuh),
// in a translation unit of its own so that the build compiles it beside the per-class kernels.
#include "sosfilt_batch.cuh"

namespace sosk {

// One persistent kernel for the whole batch: every class of the batch (section count and b0
// handling) has its own ticket counter and tile queue, and block b starts on the class whose share
// of the grid holds it (shares in proportion to the classes' work), then takes every other class
// that still has tiles, so no block idles while any class has work and the classes' tails overlap.
// A block only ever waits on tiles of its current class that were drawn before its own, which are
// held by resident blocks (the grid is persistent), so the per-signal lookback chains cannot wait
// on a block that is not running.
__global__ void __launch_bounds__((kBatchW + 1) * 32, 1) sos_batch_all_kernel(const __grid_constant__ BatchAllParams p) {
    extern __shared__ float4 smem4[];
    int first = 0;
    while (first + 1 < p.n_classes && static_cast<int>(blockIdx.x) >= p.blk_off[first + 1]) ++first;
    for (int i = 0; i < p.n_classes; ++i) {
        const int c = (first + i) % p.n_classes;
        const BatchQueue &q = p.q[c];
        switch (p.code[c]) {
#define SOSK_BATCH_CASE(k)                                                                                   \
    case 2 * (k - 1): {                                                                                      \
        const BatchParams<k> bp{q.sigs, q.tile_sig, q.n_tiles, q.desc, q.ticket, q.ticket_base, q.epoch,     \
                                p.status, p.spin_budget};                                                    \
        batch_body<k, false>(bp, smem4);                                                                     \
    } break;                                                                                                 \
    case 2 * (k - 1) + 1: {                                                                                  \
        const BatchParams<k> bp{q.sigs, q.tile_sig, q.n_tiles, q.desc, q.ticket, q.ticket_base, q.epoch,     \
                                p.status, p.spin_budget};                                                    \
        batch_body<k, true>(bp, smem4);                                                                      \
    } break;
            SOSK_BATCH_CASE(1) SOSK_BATCH_CASE(2) SOSK_BATCH_CASE(3) SOSK_BATCH_CASE(4)
            SOSK_BATCH_CASE(5) SOSK_BATCH_CASE(6) SOSK_BATCH_CASE(7) SOSK_BATCH_CASE(8)
#undef SOSK_BATCH_CASE
            default: break;
        }
        __syncthreads();  // every warp of the block is done with this class's shared state
    }
}


namespace {
KernelOnce g_once_all;

// the largest class's shared memory (eight sections)
constexpr size_t kBatchAllSmem = batch_smem_bytes<8>();

}  // namespace

cudaError_t launch_batch_all(const BatchAllParams &p, long long grid, cudaStream_t s) {
    cudaError_t e = raise_smem_once(g_once_all, sos_batch_all_kernel, kBatchAllSmem);
    if (e != cudaSuccess) return e;
    sos_batch_all_kernel<<<static_cast<unsigned>(grid), (kBatchW + 1) * 32, kBatchAllSmem, s>>>(p);
    return cudaGetLastError();
}

int batch_all_blocks_per_sm() {
    return blocks_per_sm_once(g_once_all, sos_batch_all_kernel, (kBatchW + 1) * 32, kBatchAllSmem);
}

}  // namespace sosk
