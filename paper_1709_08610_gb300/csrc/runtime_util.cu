// Host-side runtime helpers shared by the launchers.
#include <mutex>
#include <map>
#include <utility>

#include "internal.cuh"

namespace retina {

// SM count of the current device, looked up once per device.
int sm_count() {
    constexpr int kMax = 64;
    static std::mutex mu;
    static int n_of[kMax] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    int *slot = (dev >= 0 && dev < kMax) ? &n_of[dev] : nullptr;
    if (slot && *slot > 0) return *slot;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) cudaGetLastError();
    if (n <= 0) n = 1;
    if (slot) *slot = n;
    return n;
}

// The current device's opt-in limit of dynamic shared memory per block,
// looked up once per device.
int max_dynamic_smem() {
    constexpr int kMax = 64;
    static std::mutex mu;
    static int v_of[kMax] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    int *slot = (dev >= 0 && dev < kMax) ? &v_of[dev] : nullptr;
    if (slot && *slot > 0) return *slot;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) cudaGetLastError();
    if (v <= 0) v = 48 * 1024;
    if (slot) *slot = v;
    return v;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (the
// launch's own need, so that static + dynamic stays within the device's
// opt-in limit; the default limit counts static memory too, so it is raised
// even below 48 KB).  A failed request leaves no sticky error behind.
// Function attributes belong to a device's context, so the record of what was
// set is kept per (device, kernel).
cudaError_t ensure_dynamic_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    std::lock_guard<std::mutex> lock(mu);
    const std::pair<int, const void *> key(dev, func);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess)  // prefer shared memory over L1 so several such CTAs fit on an SM
        err = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err;
    }
    done[key] = bytes;
    return cudaSuccess;
}

}  // namespace retina
