// retina_grid_maxima_static: the grid-maxima selection with its scratch in a
// fixed device array owned by the library, for callers that cannot allocate
// device memory themselves (see include/retina.h).
//
// The selection needs two int32 per block of 2048 cells per event (block
// counts and their exclusive scan).  Those live in g_static_maxima_scratch,
// a file-scope __device__ array every GPU that loads the library holds until
// the process exits.  Host code must not pass the array's name to a kernel:
// on the host it is only a stand-in symbol.  The device address is obtained
// once per device with cudaGetSymbolAddress, with that device current, and
// cached.
#include <mutex>

#include "internal.cuh"

namespace retina {

static __device__ __align__(256) int32_t g_static_maxima_scratch[RETINA_STATIC_SCRATCH_BYTES / sizeof(int32_t)];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static int32_t *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on the
// first call per device).  Returns nullptr if the runtime cannot resolve it.
static int32_t *static_scratch_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_static_maxima_scratch);
        if (err != cudaSuccess || !p) return nullptr;
        g_static_ptr[dev] = static_cast<int32_t *>(p);
    }
    return g_static_ptr[dev];
}

}  // namespace retina

using namespace retina;

extern "C" int retina_grid_maxima_static(const float *R, int32_t n_events, const retina_grid *g, float R0,
                                         int32_t *max_idx, float *max_theta, float *max_R, int32_t *n_max, int32_t K,
                                         void *stream) {
    // the per-event launches put events on gridDim.y (at most 65535)
    if (n_events < 0 || n_events > 65535 || !g || isnan(R0) || K < 1) return RETINA_EINVAL;
    for (int a = 0; a < 2; ++a)
        if (!isfinite(g->lo[a]) || !(isfinite(g->step[a]) && g->step[a] > 0.f) || g->n[a] <= 0) return RETINA_EINVAL;
    if ((int64_t)g->n[0] * (int64_t)g->n[1] > (int64_t)INT32_MAX) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!R || !max_idx || !max_theta || !max_R || !n_max) return RETINA_EINVAL;
    // counts and offsets: 2 int32 per block per event
    if (maxima_ordered_ws_bytes(n_events, g) > (size_t)RETINA_STATIC_SCRATCH_BYTES) return RETINA_ENOSPACE;
    int32_t *scratch = static_scratch_for_current_device();
    if (!scratch) return RETINA_ECUDA;
    // Every call overwrites the counts of all its blocks and then all their
    // offsets before reading them, so no part of the scratch has to start at
    // zero and nothing from a previous call is read.
    return launch_grid_maxima_ordered(R, n_events, g, R0, max_idx, max_theta, max_R, n_max, K, scratch,
                                      (cudaStream_t)stream) == cudaSuccess
               ? RETINA_OK
               : RETINA_ECUDA;
}
