// The single persistent kernel over every class of a batch (sos_batch_all_kernel), with the bodies
// of every class (batch_entry, sosfilt_batch.cuh).
#include "sosfilt_batch.cuh"

namespace sosk {

// One persistent kernel for the whole batch: every class of the batch (tile geometry, section count
// and b0 handling) has its own ticket counter and tile queue, and block b starts on the class whose
// share of the grid holds it (shares in proportion to the classes' work), then takes every other
// class that still has tiles, so no block idles while any class has work and the classes' tails
// overlap.  A block only ever waits on tiles of its current class that were drawn before its own,
// which are held by resident blocks (the grid is persistent), so the per-signal lookback chains
// cannot wait on a block that is not running.  Both geometries use blocks of kBatchW + 1 warps.
__global__ void __launch_bounds__((kBatchW + 1) * 32, 1) sos_batch_all_kernel(const __grid_constant__ BatchAllParams p) {
    extern __shared__ float4 smem4[];
    int first = 0;
    while (first + 1 < p.n_classes && static_cast<int>(blockIdx.x) >= p.blk_off[first + 1]) ++first;
    for (int i = 0; i < p.n_classes; ++i) {
        const int c = (first + i) % p.n_classes;
        const BatchQueue &q = p.q[c];
        switch (p.code[c]) {
#define SOSK_BATCH_CASE(g, k, nm)                                                                             \
    case batch_class(g, k, nm): {                                                                             \
        const BatchParams<k> bp{q.sigs, q.tile_sig, q.n_tiles, q.desc, q.ticket, q.ticket_base, q.epoch,      \
                                p.status, p.spin_budget};                                                     \
        batch_entry<k, nm, batch_geom_n(g)>(bp, smem4);                                                       \
    } break;
#define SOSK_BATCH_K(g, k) SOSK_BATCH_CASE(g, k, false) SOSK_BATCH_CASE(g, k, true)
#define SOSK_BATCH_G(g) SOSK_BATCH_K(g, 1) SOSK_BATCH_K(g, 2) SOSK_BATCH_K(g, 3) SOSK_BATCH_K(g, 4) \
    SOSK_BATCH_K(g, 5) SOSK_BATCH_K(g, 6) SOSK_BATCH_K(g, 7) SOSK_BATCH_K(g, 8)
            SOSK_BATCH_G(0) SOSK_BATCH_G(1)
#undef SOSK_BATCH_G
#undef SOSK_BATCH_K
#undef SOSK_BATCH_CASE
            default: break;
        }
        __syncthreads();  // every warp of the block is done with this class's shared state
    }
}


namespace {
KernelOnce g_once_all;

// the largest class's shared memory (eight sections, 64 samples per lane)
constexpr size_t kBatchAllSmem = batch_smem_bytes<8, kBatchN>();
static_assert(batch_smem_bytes<8, kBatchNs>() <= kBatchAllSmem, "the wide geometry bounds the shared memory");

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
