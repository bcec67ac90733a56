// Cluster the converged points and keep the best of each cluster above R0
// (Algorithm 1, its last two lines), on the GPU, one CTA per event.
//
// Sequential definition: visit the candidates by decreasing R (equal R:
// lower point index first) and keep one when every point kept before it is at
// least merge_cells away in max_a |dtheta_a| / step_a.
//
// Parallel evaluation of exactly that definition:
//   1. filter candidates into shared memory (status <= 1, finite, inside the
//      box, R >= R0) with 64-bit keys (~order(R), index);
//   2. bitonic sort -> rank order;
//   3. bucket the candidates on a grid of cells slightly wider than the merge
//      distance (so any two conflicting candidates lie in adjacent buckets)
//      and sort (bucket row, bucket column, rank);
//   4. resolve in rounds: an undecided candidate is rejected as soon as a
//      lower-ranked conflicting candidate is kept, kept once every
//      lower-ranked conflicting candidate is rejected; the lowest undecided
//      rank always resolves, so rounds end;
//   5. write the kept ones in rank order.
// Conflict tests are exact: |a - b| < c is decided without rounding (c =
// merge_cells * step is exact for power-of-two steps), see abs_diff_lt.
#include "internal.cuh"

namespace retina {

constexpr int EX_THREADS = 1024;
constexpr int BUCKET_BITS = 21;
constexpr int RANK_BITS = 22;

// Exact test |a - b| < c for finite floats and c > 0 representable.
// fl() is monotone and c is representable, so |fl(a-b)| < c or > c decides
// it; on |fl(a-b)| == c the TwoSum error term says on which side a-b lies.
__device__ __forceinline__ bool abs_diff_lt(float a, float b, float c) {
    const float s = __fsub_rn(a, b);
    const float as = fabsf(s);
    if (as < c) return true;
    if (as > c) return false;
    const float nb = -b;
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(nb, bb));
    return s > 0.f ? (err < 0.f) : (err > 0.f);
}

__device__ void bitonic_sort(uint64_t *keys, int C) {
    for (int k = 2; k <= C; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < C; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sort keys[0, C) in place (C a power of two, all EX_THREADS threads call it):
// from 1024 keys on, in registers (bitonic_sort_regs, keys as its exchange
// buffer); shorter runs with the plain shared-memory network.
template <int R>
__device__ __forceinline__ void sort_keys_regs(uint64_t *keys) {
    uint64_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = keys[threadIdx.x * R + r];
    __syncthreads();
    bitonic_sort_regs<uint64_t, R, EX_THREADS>(v, keys);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) keys[threadIdx.x * R + r] = v[r];
    __syncthreads();
}

__device__ void sort_keys(uint64_t *keys, int C) {
    if (C == EX_THREADS)
        sort_keys_regs<1>(keys);
    else if (C == 2 * EX_THREADS)
        sort_keys_regs<2>(keys);
    else if (C == 4 * EX_THREADS)
        sort_keys_regs<4>(keys);
    else if (C == 8 * EX_THREADS)
        sort_keys_regs<8>(keys);
    else
        bitonic_sort(keys, C);
}

__device__ __forceinline__ int lower_bound_u64(const uint64_t *keys, int n, uint64_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Points have D coordinates (2: the two-parameter models, 4: (x0, y0, t_x,
// t_y)); the box and the buckets are on the last two (the grid's axes).
struct ExtractParams {
    float lo0, lo1, hi0, hi1;
    float c[4];      // merge distance per coordinate: merge_cells * step (or unit)
    float w0, w1;    // bucket width of the last two coordinates (slightly above c)
    float R0;
    int n_points, K, cap;
};

// Conflict of two points: closer than the merge distance in every coordinate.
template <int D>
__device__ __forceinline__ bool conflict(const float *a, const float *b, const ExtractParams &prm) {
    bool c = true;
#pragma unroll
    for (int d = 0; d < D; ++d) c = c && abs_diff_lt(a[d], b[d], prm.c[d]);
    return c;
}

// GWS: the candidate arrays (keys, coordinates, sources, states) of event e
// live in the caller's workspace at e * ws_stride instead of shared memory
// (events with more points than shared memory holds); the algorithm and its
// result are the same.
template <int D, bool GWS>
__global__ void __launch_bounds__(EX_THREADS)
extract_tracks_kernel(const float *__restrict__ theta, const float *__restrict__ R, const uint8_t *__restrict__ status,
                      const int32_t *__restrict__ n_valid, ExtractParams prm, float *__restrict__ tracks,
                      float *__restrict__ track_R, int32_t *__restrict__ track_src, int32_t *__restrict__ n_tracks,
                      unsigned char *__restrict__ ws, int64_t ws_stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int cap = prm.cap;
    unsigned char *store = GWS ? ws + (int64_t)blockIdx.x * ws_stride : smem;
    uint64_t *keys = reinterpret_cast<uint64_t *>(store);
    float *th = reinterpret_cast<float *>(keys + cap);  // [D][cap]
    int32_t *src = reinterpret_cast<int32_t *>(th + D * cap);
    volatile uint8_t *state = reinterpret_cast<uint8_t *>(src + cap);
    __shared__ int nc_s;
    __shared__ int warp_tot[EX_THREADS / 32];
    __shared__ int run;

    pdl_wait();  // may be launched while the kernel producing its points finishes
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int n = prm.n_points;
    if (n_valid) {
        const int v = n_valid[e];
        n = v < n ? (v > 0 ? v : 0) : n;
    }
    const int64_t base = (int64_t)e * prm.n_points;
    if (tid == 0) nc_s = 0;
    __syncthreads();
    // 1. filter; a thread issues the loads of its FU points together (latency-bound otherwise)
    constexpr int FU = 8;
    for (int i0 = 0; i0 < n; i0 += FU * EX_THREADS) {
        float r[FU], a0[FU], a1[FU];
        bool fin[FU];
        uint8_t sv[FU];
#pragma unroll
        for (int u = 0; u < FU; ++u) {
            const int i = i0 + u * EX_THREADS + tid;
            r[u] = a0[u] = a1[u] = 0.f;
            fin[u] = true;
            sv[u] = 0;
            if (i < n) {
                const int64_t o = base + i;
                r[u] = R[o];
                a0[u] = theta[D * o + D - 2];
                a1[u] = theta[D * o + D - 1];
#pragma unroll
                for (int d = 0; d < D - 2; ++d) fin[u] = fin[u] && isfinite(theta[D * o + d]);
                if (status) sv[u] = status[o];
            }
        }
#pragma unroll
        for (int u = 0; u < FU; ++u) {
            const int i = i0 + u * EX_THREADS + tid;
            const bool ok = i < n && fin[u] && isfinite(r[u]) && isfinite(a0[u]) && isfinite(a1[u]) &&
                            (r[u] >= prm.R0) && sv[u] <= 1 && a0[u] >= prm.lo0 && a0[u] < prm.hi0 &&
                            a1[u] >= prm.lo1 && a1[u] < prm.hi1;
            if (ok) {
                const int pos = atomicAdd(&nc_s, 1);
                keys[pos] = ((uint64_t)(~float_order_key(r[u])) << 32) | (uint32_t)i;
            }
        }
    }
    __syncthreads();
    const int nc = nc_s;
    if (nc <= 64) {
        // few candidates: one warp applies the sequential definition directly -
        // rank order by a register sort, then ranks in order, each kept unless it
        // conflicts with a kept one (lane l tests ranks l and l + 32)
        if (warp != 0) return;
        uint64_t v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) v[q] = 2 * lane + q < nc ? keys[2 * lane + q] : ~0ull;
        bitonic_sort_regs<uint64_t, 2, 32>(v, keys);
        // rank r = 2 lane + q holds v[q]; lane l keeps ranks l and l + 32 for the tests
        float a[2][D];
        int si[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = lane + 32 * h;  // rank r sits in lane r / 2, slot r % 2
            const uint64_t k0 = __shfl_sync(0xffffffffu, v[0], r >> 1), k1 = __shfl_sync(0xffffffffu, v[1], r >> 1);
            const uint64_t kr = (r & 1) ? k1 : k0;
            si[h] = (int)(uint32_t)kr;
#pragma unroll
            for (int d = 0; d < D; ++d) a[h][d] = 0.f;
            if (r < nc) {
                const int64_t o = base + si[h];
#pragma unroll
                for (int d = 0; d < D; ++d) a[h][d] = theta[D * o + d];
            }
        }
        unsigned kept0 = 0u, kept1 = 0u;  // bit l: rank l (kept0) or l + 32 (kept1) kept
        for (int r = 0; r < nc; ++r) {
            const int h = r >> 5, l = r & 31;
            float b[D];
#pragma unroll
            for (int d = 0; d < D; ++d) b[d] = __shfl_sync(0xffffffffu, h ? a[1][d] : a[0][d], l);
            const bool c0 = ((kept0 >> lane) & 1u) && conflict<D>(a[0], b, prm);
            const bool c1 = ((kept1 >> lane) & 1u) && conflict<D>(a[1], b, prm);
            if (!__any_sync(0xffffffffu, c0 || c1)) {
                if (h) kept1 |= 1u << l;
                else kept0 |= 1u << l;
            }
        }
        // kept ranks in rank order
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(((h ? kept1 : kept0) >> lane) & 1u)) continue;
            const int pos = (h ? __popc(kept0) : 0) + __popc((h ? kept1 : kept0) & ((1u << lane) - 1u));
            if (pos < prm.K) {
                const int64_t o = (int64_t)e * prm.K + pos;
#pragma unroll
                for (int d = 0; d < D; ++d) tracks[D * o + d] = a[h][d];
                track_R[o] = R[base + si[h]];
                if (track_src) track_src[o] = si[h];
            }
        }
        if (lane == 0) n_tracks[e] = __popc(kept0) + __popc(kept1);
        return;
    }
    int C = 1;
    while (C < nc) C <<= 1;
    for (int i = nc + tid; i < C; i += EX_THREADS) keys[i] = ~0ull;
    __syncthreads();
    // 2. rank order
    sort_keys(keys, C);
    for (int r = tid; r < nc; r += EX_THREADS) {
        const int i = (int)(uint32_t)keys[r];
        const int64_t o = base + i;
#pragma unroll
        for (int d = 0; d < D; ++d) th[d * cap + r] = theta[D * o + d];
        src[r] = i;
        state[r] = 0;
    }
    __syncthreads();
    const float *thb0 = th + (D - 2) * cap, *thb1 = th + (D - 1) * cap;  // the bucketed coordinates
    // 3. buckets
    const uint64_t bmax = (1ull << BUCKET_BITS) - 1;
    for (int r = tid; r < C; r += EX_THREADS) {
        if (r < nc) {
            uint64_t b0 = (uint64_t)fminf(fmaxf(floorf((thb0[r] - prm.lo0) / prm.w0), 0.f), (float)bmax);
            uint64_t b1 = (uint64_t)fminf(fmaxf(floorf((thb1[r] - prm.lo1) / prm.w1), 0.f), (float)bmax);
            keys[r] = (b1 << (BUCKET_BITS + RANK_BITS)) | (b0 << RANK_BITS) | (uint64_t)r;
        } else {
            keys[r] = ~0ull;
        }
    }
    __syncthreads();
    sort_keys(keys, C);
    // 4. rounds
    for (int round = 0; round <= nc + 1; ++round) {
        bool undecided = false;
        for (int r = tid; r < nc; r += EX_THREADS) {
            if (state[r] != 0) continue;
            float ar[D];
#pragma unroll
            for (int d = 0; d < D; ++d) ar[d] = th[d * cap + r];
            const int64_t b0 = (int64_t)fminf(fmaxf(floorf((ar[D - 2] - prm.lo0) / prm.w0), 0.f), (float)bmax);
            const int64_t b1 = (int64_t)fminf(fmaxf(floorf((ar[D - 1] - prm.lo1) / prm.w1), 0.f), (float)bmax);
            bool rejected = false, blocked = false;
            for (int dy = -1; dy <= 1 && !rejected; ++dy) {
                const int64_t row = b1 + dy;
                if (row < 0 || row > (int64_t)bmax) continue;
                const int64_t c_lo = b0 > 0 ? b0 - 1 : 0;
                const int64_t c_hi = b0 + 2;  // exclusive
                // keys of columns [c_lo, c_hi) in this row; a column past the last
                // one carries into the next row, which is the end of this row
                const uint64_t k_lo = ((uint64_t)row << (BUCKET_BITS + RANK_BITS)) + ((uint64_t)c_lo << RANK_BITS);
                const uint64_t k_hi = ((uint64_t)row << (BUCKET_BITS + RANK_BITS)) +
                                      ((uint64_t)(c_hi <= (int64_t)bmax ? c_hi : bmax + 1) << RANK_BITS);
                const int q0 = lower_bound_u64(keys, nc, k_lo);
                const int q1 = lower_bound_u64(keys, nc, k_hi);
                for (int q = q0; q < q1; ++q) {
                    const int rj = (int)(keys[q] & ((1ull << RANK_BITS) - 1));
                    if (rj >= r) continue;
                    float bj[D];
#pragma unroll
                    for (int d = 0; d < D; ++d) bj[d] = th[d * cap + rj];
                    if (!conflict<D>(ar, bj, prm)) continue;
                    const uint8_t sj = state[rj];
                    if (sj == 1) {
                        rejected = true;
                        break;
                    }
                    if (sj == 0) blocked = true;
                }
            }
            if (rejected)
                state[r] = 2;
            else if (!blocked)
                state[r] = 1;
            else
                undecided = true;
        }
        if (!__syncthreads_or(undecided)) break;
    }
    // 5. output in rank order
    if (tid == 0) run = 0;
    __syncthreads();
    for (int r0 = 0; r0 < nc; r0 += EX_THREADS) {
        const int r = r0 + tid;
        const bool kept = r < nc && state[r] == 1;
        const unsigned bal = __ballot_sync(0xffffffffu, kept);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < EX_THREADS / 32; ++w) {
            const int v = warp_tot[w];
            before += (w < warp) ? v : 0;
            tot += v;
        }
        if (kept) {
            const int pos = run + before + __popc(bal & ((1u << lane) - 1u));
            if (pos < prm.K) {
                const int64_t o = (int64_t)e * prm.K + pos;
#pragma unroll
                for (int d = 0; d < D; ++d) tracks[D * o + d] = th[d * cap + r];
                track_R[o] = R[base + src[r]];
                if (track_src) track_src[o] = src[r];
            }
        }
        __syncthreads();
        if (tid == 0) run += tot;
        __syncthreads();
    }
    if (tid == 0) n_tracks[e] = run;
}

size_t extract_smem_bytes(int n_points, int dims) {
    int64_t C = 1;
    while (C < n_points) C <<= 1;
    return (size_t)C * (sizeof(uint64_t) + (size_t)dims * sizeof(float) + sizeof(int32_t) + 1) + 16;
}

// Workspace of the global-memory form: per event the same arrays, 256-aligned.
size_t extract_ws_stride(int n_points, int dims) { return (extract_smem_bytes(n_points, dims) + 255) / 256 * 256; }

// merge[d]: the merge distance of coordinate d; box on the last two.
template <int D>
static cudaError_t launch_extract_d(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                                    int n_events, int n_points, const retina_grid *box, float R0, const float *merge,
                                    float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int K,
                                    cudaStream_t st, void *ws = nullptr) {
    const bool gws = ws != nullptr;
    const size_t smem = gws ? 0 : extract_smem_bytes(n_points, D);
    if (!gws) {
        cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(extract_tracks_kernel<D, false>), smem);
        if (aerr != cudaSuccess) return aerr;
    }
    ExtractParams prm{};
    prm.lo0 = box->lo[0];
    prm.lo1 = box->lo[1];
    prm.hi0 = box->lo[0] + (float)box->n[0] * box->step[0];
    prm.hi1 = box->lo[1] + (float)box->n[1] * box->step[1];
    for (int d = 0; d < D; ++d) prm.c[d] = merge[d];
    prm.w0 = prm.c[D - 2] * 1.015625f;
    prm.w1 = prm.c[D - 1] * 1.015625f;
    prm.R0 = R0;
    prm.n_points = n_points;
    prm.K = K;
    int C = 1;
    while (C < n_points) C <<= 1;
    prm.cap = C;
    PrioLaunch L(dim3(n_events), dim3(EX_THREADS), smem, st, true);
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    const int64_t stride = gws ? (int64_t)extract_ws_stride(n_points, D) : 0;
    const cudaError_t lerr =
        gws ? cudaLaunchKernelEx(&L.cfg, extract_tracks_kernel<D, true>, theta, R, status, n_valid, prm, tracks,
                                 track_R, track_src, n_tracks, wsb, stride)
            : cudaLaunchKernelEx(&L.cfg, extract_tracks_kernel<D, false>, theta, R, status, n_valid, prm, tracks,
                                 track_R, track_src, n_tracks, wsb, stride);
    count_launches(1);
    return lerr != cudaSuccess ? lerr : cudaGetLastError();
}

cudaError_t launch_extract_tracks(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                                  int n_events, int n_points, const retina_grid *box, float R0, float merge_cells,
                                  float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int K,
                                  cudaStream_t st, void *ws) {
    const float merge[2] = {merge_cells * box->step[0], merge_cells * box->step[1]};
    // shared memory holds up to RETINA_MAX_EXTRACT_POINTS points; beyond that the workspace
    return launch_extract_d<2>(theta, R, status, n_valid, n_events, n_points, box, R0, merge, tracks, track_R,
                               track_src, n_tracks, K, st, n_points > RETINA_MAX_EXTRACT_POINTS ? ws : nullptr);
}

cudaError_t launch_extract_tracks4(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                                   int n_events, int n_points, const retina_grid *slope_box, const float unit[4],
                                   float R0, float merge_units, float *tracks, float *track_R, int32_t *track_src,
                                   int32_t *n_tracks, int K, cudaStream_t st) {
    const float merge[4] = {merge_units * unit[0], merge_units * unit[1], merge_units * unit[2],
                            merge_units * unit[3]};
    return launch_extract_d<4>(theta, R, status, n_valid, n_events, n_points, slope_box, R0, merge, tracks, track_R,
                               track_src, n_tracks, K, st);
}

}  // namespace retina
