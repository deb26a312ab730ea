// sos_filter_run_noalloc: the default filter run (PH factorization) with its scratch memory (lookback
// descriptors and ticket counter) in one file-scope device array instead of library
// allocations.  For callers that cannot allocate device memory while they filter: a real-time
// thread (an audio or radio receive loop) must not call cudaMalloc/cudaFree, which can block
// and synchronize the device, and some applications hand out all device memory at start-up.
// Such callers create the filter object once during set-up and then filter with this entry
// point, which allocates nothing: no cudaMalloc, cudaFree or other allocating CUDA routine, and no
// host heap allocation.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "sosfilt.h"
#include "sosfilt_internal.h"

namespace sosk {
int filter_device(const sos_filter *f);
sos_status run_lane_scratch(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf,
                            cudaStream_t s, const Scratch &sc, unsigned (*next_epoch)(int, cudaStream_t));
}  // namespace sosk

namespace {

// Word 0: ticket counter; words 32..: lookback descriptors (tag << 32 | float bits).  Sized for
// SOS_NOALLOC_MAX_SAMPLES samples per call (PH tiles of 7 x 2048 samples, two slots of up to 16
// words each).
constexpr size_t kDescWords =
    (static_cast<size_t>(SOS_NOALLOC_MAX_SAMPLES) / (sosk::kLaneW * sosk::kL * 64) + 1) * 2 * 2 * sosk::kMaxPass;
constexpr size_t kScratchWords = 32 + kDescWords;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
unsigned long long *g_ptr[64] = {nullptr};  // device address of g_noalloc_scratch, per device
unsigned g_epoch[64] = {0};                 // last epoch used on that device (tags are never 0)

// Tag of the next pass on device dev (called with g_mu held): 1 .. 2^30 - 1, never 0.  Every pass
// clears the descriptors it uses before its launch, so a tag only has to differ from 0.
unsigned next_epoch_dev(int dev, cudaStream_t) {
    g_epoch[dev] = g_epoch[dev] % 0x3fffffffu + 1;
    return g_epoch[dev];
}

}  // namespace

extern "C" sos_status sos_filter_run_noalloc(sos_filter *f, const float *x_dev, float *y_dev, int64_t n,
                                             const float *zi_dev, float *zf_dev, void *stream) {
    if (!f || n < 0) return SOS_EINVAL;
    if (n > SOS_NOALLOC_MAX_SAMPLES) return SOS_EBUDGET;
    const int dev = sosk::filter_device(f);
    if (dev < 0 || dev >= 64) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaSetDevice(dev) != cudaSuccess) return SOS_ECUDA;
    if (!g_ptr[dev]) {
        // one-time set-up on this device, with it current: the array's device address
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SOS_ECUDA;
        g_ptr[dev] = static_cast<unsigned long long *>(ptr);
    }
    sosk::Scratch sc;
    sc.ticket = g_ptr[dev];
    sc.desc = g_ptr[dev] + 32;
    sc.desc_words = kDescWords;
    return sosk::run_lane_scratch(f, x_dev, y_dev, n, zi_dev, zf_dev, static_cast<cudaStream_t>(stream), sc,
                                  next_epoch_dev);
}
