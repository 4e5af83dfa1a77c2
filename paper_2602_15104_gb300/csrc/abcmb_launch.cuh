// Host-side launch helper shared by the kernels that take large dynamic
// shared memory.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <map>
#include <utility>

namespace abcmb {

// Opt a kernel in to the largest dynamic shared memory the device allows,
// once per (kernel, device).  The attribute is global state of the kernel,
// which the driver orders against that kernel's launches still in flight on
// other streams: set on every launch it would serialise concurrent callers.
// Returns the bytes of dynamic shared memory the kernel may now use, or -1.
inline long smem_optin(const void *func)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    static std::mutex m;
    static std::map<std::pair<const void *, int>, long> done;
    std::lock_guard<std::mutex> lock(m);
    const auto it = done.find({func, dev});
    if (it != done.end()) return it->second;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return -1;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return -1;
    const long avail = (long)optin - (long)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail) != cudaSuccess)
        return -1;
    done[{func, dev}] = avail;
    return avail;
}

} // namespace abcmb
