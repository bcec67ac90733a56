// Host-side runtime helpers shared by the launchers.
#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace retina {

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        if (n <= 0) n = 1;
    }
    return n;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (the
// launch's own need, so that static + dynamic stays within the device's
// opt-in limit; the default limit counts static memory too, so it is raised
// even below 48 KB).  A failed request leaves no sticky error behind.
cudaError_t ensure_dynamic_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void *, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(func);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess)  // prefer shared memory over L1 so several such CTAs fit on an SM
        err = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err;
    }
    done[func] = bytes;
    return cudaSuccess;
}

}  // namespace retina
