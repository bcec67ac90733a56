// Opt-in count of the work the response kernels actually perform (pairs of
// (point or cell, hit) evaluated, after exact block skipping), for rooflines.
// Kernels receive the counters' device address as an argument (nullptr when
// counting is off) and add to them once per CTA or warp.
#include <atomic>
#include <mutex>

#include "internal.cuh"

namespace retina {

static __device__ unsigned long long g_work[RETINA_WORK_KINDS];
static std::atomic<int> g_counting{0};
static std::mutex g_work_mu;
static unsigned long long *g_work_ptr[64] = {nullptr};

unsigned long long *work_counters() {
    if (!g_counting.load(std::memory_order_relaxed)) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_work_mu);
    if (!g_work_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_work) != cudaSuccess) return nullptr;
        g_work_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    return g_work_ptr[dev];
}

// Device-side error flag of the library: set (to 1) by a kernel whose
// bounded wait expired; read and cleared with retina_device_error.
static __device__ int32_t g_dev_error;
static int32_t *g_err_ptr[64] = {nullptr};

int32_t *device_error_flag() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_work_mu);
    if (!g_err_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dev_error) != cudaSuccess) return nullptr;
        g_err_ptr[dev] = static_cast<int32_t *>(p);
    }
    return g_err_ptr[dev];
}

}  // namespace retina

using namespace retina;

extern "C" int retina_device_error(int32_t *flag, int32_t reset) {
    if (flag) {
        int32_t v = 0;
        if (cudaMemcpyFromSymbol(&v, g_dev_error, sizeof(v)) != cudaSuccess) return RETINA_ECUDA;
        *flag = v;
    }
    if (reset) {
        const int32_t zero = 0;
        if (cudaMemcpyToSymbol(g_dev_error, &zero, sizeof(zero)) != cudaSuccess) return RETINA_ECUDA;
    }
    return RETINA_OK;
}

extern "C" int retina_work_counters(int32_t enable, int32_t reset, uint64_t *out) {
    if (reset) {
        const unsigned long long zero[RETINA_WORK_KINDS] = {0, 0, 0, 0};
        if (cudaMemcpyToSymbol(g_work, zero, sizeof(zero)) != cudaSuccess) return RETINA_ECUDA;
    }
    if (out) {
        unsigned long long v[RETINA_WORK_KINDS];
        if (cudaMemcpyFromSymbol(v, g_work, sizeof(v)) != cudaSuccess) return RETINA_ECUDA;
        for (int i = 0; i < RETINA_WORK_KINDS; ++i) out[i] = v[i];
    }
    if (enable >= 0) g_counting = enable ? 1 : 0;
    return RETINA_OK;
}
