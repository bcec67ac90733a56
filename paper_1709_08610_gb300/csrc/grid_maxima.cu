// Selection of activated units on the grid (Section 2, steps 3-4 of the grid
// algorithm): a unit is selected when R >= R0 and it beats every existing
// neighbour of its 3 x 3 neighbourhood in the order (R, -linear index).
//
// Deterministic, ordered compaction in three launches:
//   1. maxima_pass_kernel<false>: count selected units per block of cells;
//   2. maxima_scan_kernel: exclusive scan of the block counts per event
//      (also writes the event's total);
//   3. maxima_pass_kernel<true>: re-test each unit and write the selected ones
//      at (block offset + rank within the block), i.e. in increasing linear
//      index, keeping only the first K per event.
#include "internal.cuh"

namespace retina {

constexpr int MAX_THREADS = 256, MAX_PER_THREAD = 8, MAX_BLOCK_CELLS = MAX_THREADS * MAX_PER_THREAD;

__device__ __forceinline__ bool is_selected(const float *__restrict__ R, int n0, int n1, int64_t c, float R0) {
    const int i1 = (int)(c / n0), i0 = (int)(c - (int64_t)i1 * n0);
    const float v = R[c];
    if (!(v >= R0)) return false;
#pragma unroll
    for (int d1 = -1; d1 <= 1; ++d1) {
        const int j1 = i1 + d1;
        if (j1 < 0 || j1 >= n1) continue;
#pragma unroll
        for (int d0 = -1; d0 <= 1; ++d0) {
            if (d0 == 0 && d1 == 0) continue;
            const int j0 = i0 + d0;
            if (j0 < 0 || j0 >= n0) continue;
            const int64_t nb = (int64_t)j1 * n0 + j0;
            const float w = R[nb];
            const bool beats = (v > w) || (v == w && c < nb);
            if (!beats) return false;
        }
    }
    return true;
}

template <bool WRITE>
__global__ void __launch_bounds__(MAX_THREADS)
maxima_pass_kernel(const float *__restrict__ Rall, int n0, int n1, float R0, int nblk, int32_t *__restrict__ counts,
                   const int32_t *__restrict__ offsets, GridDev g, int K, int32_t *__restrict__ max_idx,
                   float *__restrict__ max_theta, float *__restrict__ max_R) {
    __shared__ int warp_tot[MAX_THREADS / 32];
    __shared__ int run;
    const int e = blockIdx.y, blk = blockIdx.x;
    const int64_t cells = (int64_t)n0 * n1;
    const float *R = Rall + (int64_t)e * cells;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t base = (int64_t)blk * MAX_BLOCK_CELLS;
    if (t == 0) run = WRITE ? offsets[(int64_t)e * nblk + blk] : 0;
    __syncthreads();
    for (int m = 0; m < MAX_PER_THREAD; ++m) {
        const int64_t c = base + (int64_t)m * MAX_THREADS + t;
        const bool sel = c < cells && is_selected(R, n0, n1, c, R0);
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < MAX_THREADS / 32; ++w) {
            const int v = warp_tot[w];
            before += (w < warp) ? v : 0;
            tot += v;
        }
        if (WRITE && sel) {
            const int pos = run + before + __popc(bal & ((1u << lane) - 1u));
            if (pos < K) {
                const int64_t o = (int64_t)e * K + pos;
                const int i1 = (int)(c / n0), i0 = (int)(c - (int64_t)i1 * n0);
                max_idx[o] = (int32_t)c;
                max_theta[2 * o + 0] = cell_centre(g.lo0, g.step0, i0);
                max_theta[2 * o + 1] = cell_centre(g.lo1, g.step1, i1);
                max_R[o] = R[c];
            }
        }
        __syncthreads();
        if (t == 0) run += tot;
        __syncthreads();
    }
    if (!WRITE && t == 0) counts[(int64_t)e * nblk + blk] = run;
}

__global__ void maxima_scan_kernel(const int32_t *__restrict__ counts, int nblk, int32_t *__restrict__ offsets,
                                   int32_t *__restrict__ n_max) {
    // one block of 1024 threads per event; chunked Hillis-Steele scan
    __shared__ int buf[1024];
    __shared__ int carry;
    const int e = blockIdx.x, t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        const int b = b0 + t;
        const int v = b < nblk ? counts[(int64_t)e * nblk + b] : 0;
        buf[t] = v;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {
            const int add = t >= d ? buf[t - d] : 0;
            __syncthreads();
            buf[t] += add;
            __syncthreads();
        }
        if (b < nblk) offsets[(int64_t)e * nblk + b] = carry + buf[t] - v;
        __syncthreads();
        if (t == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (t == 0) n_max[e] = carry;
}

int maxima_blocks(const retina_grid *g) {
    const int64_t cells = (int64_t)g->n[0] * g->n[1];
    return (int)((cells + MAX_BLOCK_CELLS - 1) / MAX_BLOCK_CELLS);
}

size_t maxima_ws_bytes(int n_events, const retina_grid *g) {
    return 2 * (size_t)n_events * (size_t)maxima_blocks(g) * sizeof(int32_t);
}

cudaError_t launch_grid_maxima(const float *R, int n_events, const retina_grid *g, float R0, int32_t *max_idx,
                               float *max_theta, float *max_R, int32_t *n_max, int K, int32_t *ws_counts,
                               cudaStream_t st) {
    const int nblk = maxima_blocks(g);
    int32_t *counts = ws_counts;
    int32_t *offsets = ws_counts + (int64_t)n_events * nblk;
    GridDev gd{g->lo[0], g->lo[1], g->step[0], g->step[1], g->n[0], g->n[1]};
    dim3 grid(nblk, n_events);
    maxima_pass_kernel<false><<<grid, MAX_THREADS, 0, st>>>(R, g->n[0], g->n[1], R0, nblk, counts, nullptr, gd, K,
                                                            nullptr, nullptr, nullptr);
    maxima_scan_kernel<<<n_events, 1024, 0, st>>>(counts, nblk, offsets, n_max);
    maxima_pass_kernel<true><<<grid, MAX_THREADS, 0, st>>>(R, g->n[0], g->n[1], R0, nblk, counts, offsets, gd, K,
                                                           max_idx, max_theta, max_R);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace retina
