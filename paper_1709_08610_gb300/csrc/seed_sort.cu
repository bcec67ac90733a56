// Spatial ordering of each event's starting points (retina_sort_seeds).
//
// Algorithm 1 treats its starting points independently, so their order is
// free.  Neighbouring points need mostly the same hit blocks, so a warp that
// searches several consecutive points (RETINA_OPT_BATCH_SEEDS_PER_WARP > 1)
// shares block tests and hit loads when the points are spatially ordered.
// Key of a point: the Hilbert index (order 9) of its position in the box
// quantised to 9 bits per axis (points outside the box clamp to the edge;
// non-finite ones get 2^18, after every finite point), over its 13-bit index
// in the chunk (chunks of 8192 points per event), so keys are distinct and
// the order is deterministic.  Consecutive Hilbert cells touch, so groups of
// consecutive points have small spans (a Morton order jumps at quadrant
// edges).
#include "internal.cuh"

namespace retina {

constexpr int SS_THREADS = 1024;
constexpr int SS_IDX_BITS = 13;
constexpr int SS_CAP = 1 << SS_IDX_BITS;

__device__ __forceinline__ uint32_t quant9(float t, float lo, float inv_ext) {
    const float q = (t - lo) * inv_ext;
    if (!(q > 0.f)) return 0u;  // also NaN
    if (!(q < 1.f)) return 511u;
    return (uint32_t)(q * 512.f) & 511u;
}

template <int R>
__device__ __forceinline__ void sort_seed_chunk(const float2 *__restrict__ seeds, int64_t base, int n, float lo0,
                                                float lo1, float inv0, float inv1, float2 *__restrict__ out,
                                                int32_t *__restrict__ perm, uint32_t *x) {
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        uint32_t key = 0xffffffffu;
        if (i < n) {
            const float2 s = seeds[base + i];
            const uint32_t m = (isfinite(s.x) && isfinite(s.y))
                                   ? hilbert_index<9>(quant9(s.x, lo0, inv0), quant9(s.y, lo1, inv1))
                                   : (1u << 18);  // after every finite point
            key = (m << SS_IDX_BITS) | (uint32_t)i;
        }
        v[r] = key;
    }
    bitonic_sort_regs<uint32_t, R, SS_THREADS>(v, x);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        if (i < n) {
            const int src = (int)(v[r] & (SS_CAP - 1));
            out[base + i] = seeds[base + src];
            if (perm) perm[base + i] = (int32_t)(base + src);
        }
    }
}

__global__ void __launch_bounds__(SS_THREADS)
sort_seeds_kernel(const float2 *__restrict__ seeds, int64_t n_seeds, const int64_t *__restrict__ off, float lo0,
                  float lo1, float inv0, float inv1, float2 *__restrict__ out, int32_t *__restrict__ perm) {
    __shared__ uint32_t x[SS_CAP];
    int64_t sb, se;
    event_range(off, n_seeds, blockIdx.x, sb, se);
    for (int64_t c0 = sb; c0 < se; c0 += SS_CAP) {
        const int n = (int)((se - c0) < SS_CAP ? (se - c0) : SS_CAP);
        if (n <= SS_THREADS)
            sort_seed_chunk<1>(seeds, c0, n, lo0, lo1, inv0, inv1, out, perm, x);
        else if (n <= 2 * SS_THREADS)
            sort_seed_chunk<2>(seeds, c0, n, lo0, lo1, inv0, inv1, out, perm, x);
        else if (n <= 4 * SS_THREADS)
            sort_seed_chunk<4>(seeds, c0, n, lo0, lo1, inv0, inv1, out, perm, x);
        else
            sort_seed_chunk<8>(seeds, c0, n, lo0, lo1, inv0, inv1, out, perm, x);
        __syncthreads();
    }
}

cudaError_t launch_sort_seeds(const float *seeds, int64_t n_seeds, const int64_t *off, int n_events,
                              const retina_grid *box, float *out, int32_t *perm, cudaStream_t st) {
    const float inv0 = (float)(1.0 / ((double)box->n[0] * (double)box->step[0]));
    const float inv1 = (float)(1.0 / ((double)box->n[1] * (double)box->step[1]));
    sort_seeds_kernel<<<n_events, SS_THREADS, 0, st>>>(reinterpret_cast<const float2 *>(seeds), n_seeds, off,
                                                      box->lo[0], box->lo[1], inv0, inv1,
                                                      reinterpret_cast<float2 *>(out), perm);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
