// Selection of activated units on the grid (Section 2, steps 3-4 of the grid
// algorithm): a unit is selected when R >= R0 and it beats every existing
// neighbour of its 3 x 3 neighbourhood in the order (R, -linear index).
// Output: the selected units of each event in increasing linear index, the
// first K of them, and the total count.
//
// Two launches (launch_grid_maxima):
//   1. maxima_detect_kernel: every unit is tested; selected ones are appended
//      to a per-event candidate list (warp-aggregated atomics, any order);
//   2. maxima_order_kernel: one CTA per event sorts its candidates by index
//      and writes the first K.  If an event has more candidates than the
//      list holds, the CTA instead walks the whole grid in index order with
//      a block-wide ordered compaction (exact, slower; the list is then not
//      used).
// The three-launch ordered compaction (launch_grid_maxima_ordered: count per
// block of cells, scan, re-test and write) serves the allocation-free entry,
// whose fixed scratch holds two integers per block instead of a list.
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

size_t maxima_ordered_ws_bytes(int n_events, const retina_grid *g) {
    return 2 * (size_t)n_events * (size_t)maxima_blocks(g) * sizeof(int32_t);
}

cudaError_t launch_grid_maxima_ordered(const float *R, int n_events, const retina_grid *g, float R0,
                                       int32_t *max_idx, float *max_theta, float *max_R, int32_t *n_max, int K,
                                       int32_t *ws_counts, cudaStream_t st) {
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

// ---------------------------------------------------------------------------
// detect + order
// ---------------------------------------------------------------------------
constexpr int CAND_CAP = 4096;          // candidates listed per event
constexpr int ORDER_THREADS = 1024;

// Four cells per thread (one 16-byte load when rows are a multiple of 4 cells
// long); the neighbourhood is read only for cells >= R0.
__global__ void __launch_bounds__(MAX_THREADS)
maxima_detect_kernel(const float *__restrict__ Rall, int n0, int n1, float R0, int32_t *__restrict__ cand_count,
                     int32_t *__restrict__ cand) {
    pdl_release();
    const int e = blockIdx.y;
    const int64_t cells = (int64_t)n0 * n1;
    const float *R = Rall + (int64_t)e * cells;
    const int lane = threadIdx.x & 31;
    const int64_t c0 = 4 * ((int64_t)blockIdx.x * MAX_THREADS + threadIdx.x);
    float v[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if ((n0 & 3) == 0 && c0 + 3 < cells) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(R + c0));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c0 + u < cells) v[u] = __ldg(R + c0 + u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t c = c0 + u;
        const bool sel = (v[u] >= R0) && c < cells && is_selected(R, n0, n1, c, R0);
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (bal == 0u) continue;
        int first = 0;
        if (lane == 0) first = atomicAdd(&cand_count[e], __popc(bal));
        first = __shfl_sync(0xffffffffu, first, 0);
        const int pos = first + __popc(bal & ((1u << lane) - 1u));
        if (sel && pos < CAND_CAP) cand[(int64_t)e * CAND_CAP + pos] = (int32_t)c;
    }
}

template <int RK>
__device__ __forceinline__ void order_candidates(const int32_t *__restrict__ cand, int n, uint32_t *x,
                                                 uint32_t (&v)[RK]) {
#pragma unroll
    for (int r = 0; r < RK; ++r) {
        const int i = threadIdx.x * RK + r;
        v[r] = i < n ? (uint32_t)cand[i] : 0xffffffffu;
    }
    bitonic_sort_regs<uint32_t, RK, ORDER_THREADS>(v, x);
}

__device__ __forceinline__ void write_maximum(const float *__restrict__ R, GridDev g, int64_t o, int64_t c,
                                              int32_t *__restrict__ max_idx, float *__restrict__ max_theta,
                                              float *__restrict__ max_R) {
    const int i1 = (int)(c / g.n0), i0 = (int)(c - (int64_t)i1 * g.n0);
    max_idx[o] = (int32_t)c;
    max_theta[2 * o + 0] = cell_centre(g.lo0, g.step0, i0);
    max_theta[2 * o + 1] = cell_centre(g.lo1, g.step1, i1);
    max_R[o] = R[c];
}

__global__ void __launch_bounds__(ORDER_THREADS)
maxima_order_kernel(const float *__restrict__ Rall, GridDev g, float R0, const int32_t *__restrict__ cand_count,
                    const int32_t *__restrict__ cand, int K, int32_t *__restrict__ max_idx,
                    float *__restrict__ max_theta, float *__restrict__ max_R, int32_t *__restrict__ n_max) {
    __shared__ uint32_t x[CAND_CAP];
    __shared__ int warp_tot[ORDER_THREADS / 32];
    pdl_wait();  // launched as a dependent of maxima_detect_kernel
    pdl_release();
    const int e = blockIdx.x, t = threadIdx.x;
    const int64_t cells = (int64_t)g.n0 * g.n1;
    const float *R = Rall + (int64_t)e * cells;
    const int total = cand_count[e];
    if (t == 0) n_max[e] = total;
    const int32_t *ce = cand + (int64_t)e * CAND_CAP;
    if (total <= 64) {
        // few candidates: one warp sorts them in registers
        if (t >= 32) return;
        uint32_t v[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) v[r] = 2 * t + r < total ? (uint32_t)ce[2 * t + r] : 0xffffffffu;
        bitonic_sort_regs<uint32_t, 2, 32>(v, x);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int q = 2 * t + r;
            if (q < total && q < K) write_maximum(R, g, (int64_t)e * K + q, v[r], max_idx, max_theta, max_R);
        }
        return;
    }
    if (total <= CAND_CAP) {
        // sorted by linear index; thread t holds ranks t RK .. t RK + RK - 1
#define RETINA_ORDER_CASE(RK)                                                          \
        {                                                                              \
            uint32_t v[RK];                                                            \
            order_candidates<RK>(ce, total, x, v);                                     \
            _Pragma("unroll") for (int r = 0; r < RK; ++r) {                           \
                const int q = t * RK + r;                                              \
                if (q < total && q < K)                                                \
                    write_maximum(R, g, (int64_t)e * K + q, v[r], max_idx, max_theta, max_R); \
            }                                                                          \
        }
        if (total <= ORDER_THREADS) RETINA_ORDER_CASE(1)
        else if (total <= 2 * ORDER_THREADS) RETINA_ORDER_CASE(2)
        else RETINA_ORDER_CASE(4)
#undef RETINA_ORDER_CASE
        return;
    }
    // overflow: ordered compaction over the whole grid, stopping after K
    const int lane = t & 31, warp = t >> 5;
    int run = 0;
    for (int64_t b0 = 0; b0 < cells && run < K; b0 += ORDER_THREADS) {
        const int64_t c = b0 + t;
        const bool sel = c < cells && is_selected(R, g.n0, g.n1, c, R0);
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < ORDER_THREADS / 32; ++w) {
            const int v = warp_tot[w];
            before += (w < warp) ? v : 0;
            tot += v;
        }
        const int pos = run + before + __popc(bal & ((1u << lane) - 1u));
        if (sel && pos < K) write_maximum(R, g, (int64_t)e * K + pos, c, max_idx, max_theta, max_R);
        run += tot;  // identical in every thread
        __syncthreads();
    }
}

size_t maxima_ws_bytes(int n_events, const retina_grid *) {
    return (size_t)n_events * (CAND_CAP + 64) * sizeof(int32_t);
}

cudaError_t launch_grid_maxima(const float *R, int n_events, const retina_grid *g, float R0, int32_t *max_idx,
                               float *max_theta, float *max_R, int32_t *n_max, int K, int32_t *ws,
                               cudaStream_t st) {
    int32_t *cand_count = ws;                                   // [E], padded to 64 ints per event
    int32_t *cand = ws + (int64_t)n_events * 64;                // [E][CAND_CAP]
    cudaError_t err = cudaMemsetAsync(cand_count, 0, (size_t)n_events * sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    GridDev gd{g->lo[0], g->lo[1], g->step[0], g->step[1], g->n[0], g->n[1]};
    const int64_t cells = (int64_t)g->n[0] * g->n[1];
    const int dblk = (int)((cells + 4 * MAX_THREADS - 1) / (4 * MAX_THREADS));
    maxima_detect_kernel<<<dim3(dblk, n_events), MAX_THREADS, 0, st>>>(R, g->n[0], g->n[1], R0, cand_count, cand);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    PrioLaunch L(dim3(n_events), dim3(ORDER_THREADS), 0, st, true);
    err = cudaLaunchKernelEx(&L.cfg, maxima_order_kernel, R, gd, R0, (const int32_t *)cand_count,
                             (const int32_t *)cand, K, max_idx, max_theta, max_R, n_max);
    count_launches(2);
    return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace retina
