/*
 * Host stand-in for the few CUDA runtime declarations the serving loop (sosfilt_server.cpp) uses,
 * so that its scheduling logic can be compiled and tested on a machine without a GPU.  Test
 * infrastructure only: "device" memory is host memory, and a stream is a worker thread running its
 * queued work in order (server_host.cpp).
 */
#pragma once
#include <cstddef>

typedef int cudaError_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2 };
typedef struct host_stream *cudaStream_t;
typedef void (*cudaHostFn_t)(void *);
enum cudaMemcpyKind { cudaMemcpyHostToDevice = 1, cudaMemcpyDeviceToHost = 2, cudaMemcpyDeviceToDevice = 3 };
#define cudaStreamNonBlocking 1
#define CUDART_CB

cudaError_t cudaSetDevice(int device);
cudaError_t cudaGetDevice(int *device);
cudaError_t cudaGetLastError(void);
cudaError_t cudaMalloc(void **ptr, size_t bytes);
cudaError_t cudaFree(void *ptr);
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind);
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *stream, unsigned flags);
cudaError_t cudaStreamSynchronize(cudaStream_t stream);
cudaError_t cudaStreamDestroy(cudaStream_t stream);
cudaError_t cudaLaunchHostFunc(cudaStream_t stream, cudaHostFn_t fn, void *arg);

// the runtime's typed convenience overload
template <class T>
cudaError_t cudaMalloc(T **ptr, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
}
