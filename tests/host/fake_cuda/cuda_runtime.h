// Stand-in for the CUDA runtime API, for building the spectrum server's host
// runtime (abcmb_server.cu) on the CPU in the tests: the types and calls the
// server uses, implemented in tests/host/server_harness.cpp over host memory.
// Copies run at once; an event reports completion only after it has been
// queried a set number of times, so the server's non-blocking retire path
// runs.  Not a model of the device.
#pragma once

#include <cstddef>

typedef enum cudaError { cudaSuccess = 0, cudaErrorNotReady = 600, cudaErrorUnknown = 999 } cudaError_t;
enum cudaMemcpyKind { cudaMemcpyHostToDevice = 1, cudaMemcpyDeviceToHost = 2 };
struct FakeStream;
struct FakeEvent;
typedef FakeStream *cudaStream_t;
typedef FakeEvent *cudaEvent_t;
#define cudaStreamNonBlocking 0x01
#define cudaEventDisableTiming 0x02

cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned flags);
cudaError_t cudaStreamDestroy(cudaStream_t s);
cudaError_t cudaStreamSynchronize(cudaStream_t s);
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned flags);
cudaError_t cudaEventDestroy(cudaEvent_t e);
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s);
cudaError_t cudaEventQuery(cudaEvent_t e);
cudaError_t cudaMallocHost(void **p, size_t bytes);
cudaError_t cudaFreeHost(void *p);
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s);
cudaError_t cudaMemcpy2DAsync(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                              cudaMemcpyKind kind, cudaStream_t s);
