/*
 * Host stand-in for the CUDA runtime declarations the library's host code (sosfilt_api.cpp) uses,
 * so that its table building, argument handling, launch planning, batching and host-buffer
 * pipeline can be compiled and tested without a GPU.  Test infrastructure only: "device" memory is
 * host memory and every stream runs its work at once, in the calling thread (api_host.cpp).
 */
#pragma once
#include <cstddef>

struct alignas(8) float2 {
    float x, y;
};
struct alignas(16) float4 {
    float x, y, z, w;
};

typedef int cudaError_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2 };
typedef struct host_stream *cudaStream_t;
typedef struct host_event *cudaEvent_t;
enum cudaMemcpyKind { cudaMemcpyHostToDevice = 1, cudaMemcpyDeviceToHost = 2, cudaMemcpyDeviceToDevice = 3 };
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount = 16 };
enum cudaStreamCaptureStatus { cudaStreamCaptureStatusNone = 0, cudaStreamCaptureStatusActive = 1 };
#define cudaStreamNonBlocking 1
#define cudaEventDisableTiming 2

cudaError_t cudaSetDevice(int device);
cudaError_t cudaGetDevice(int *device);
cudaError_t cudaGetLastError(void);
cudaError_t cudaDeviceSynchronize(void);
cudaError_t cudaDeviceGetAttribute(int *value, cudaDeviceAttr attr, int device);
cudaError_t cudaMalloc(void **ptr, size_t bytes);
cudaError_t cudaFree(void *ptr);
cudaError_t cudaMallocHost(void **ptr, size_t bytes);
cudaError_t cudaHostGetDevicePointer(void **dptr, void *hptr, unsigned flags);
cudaError_t cudaFreeHost(void *ptr);
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind);
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s = nullptr);
cudaError_t cudaMemset(void *dst, int value, size_t bytes);
cudaError_t cudaMemsetAsync(void *dst, int value, size_t bytes, cudaStream_t s = nullptr);
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *stream, unsigned flags);
cudaError_t cudaStreamSynchronize(cudaStream_t stream);
cudaError_t cudaStreamIsCapturing(cudaStream_t stream, cudaStreamCaptureStatus *status);
cudaError_t cudaStreamDestroy(cudaStream_t stream);
cudaError_t cudaStreamWaitEvent(cudaStream_t stream, cudaEvent_t event, unsigned flags = 0);
cudaError_t cudaEventCreate(cudaEvent_t *event);
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *event, unsigned flags);
cudaError_t cudaEventRecord(cudaEvent_t event, cudaStream_t stream = nullptr);
cudaError_t cudaEventSynchronize(cudaEvent_t event);
cudaError_t cudaEventDestroy(cudaEvent_t event);
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t start, cudaEvent_t end);

// the runtime's typed convenience overloads
template <class T>
cudaError_t cudaMalloc(T **ptr, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
}
template <class T>
cudaError_t cudaMallocHost(T **ptr, size_t bytes) {
    return cudaMallocHost(reinterpret_cast<void **>(ptr), bytes);
}
