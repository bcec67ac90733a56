// Spatial ordering of each event's hits plus a bounding box per block of 32,
// so that the response kernels can skip, exactly, blocks whose every term of
// Eq. 1 is zero in float32.
//
// Each hit gets a band and a spatial code.  Slope model: the band is an
// octave of |z| (from 16 mm; 7 bands) and the code, below the band, is the
// index of the hit's slopes (u, v) = (x/z, y/z), quantised to 256 levels on
// [-1, 1] (clamped at the edges), along the Hilbert curve of order 8, whose
// consecutive cells always touch (a Morton order jumps at every quadrant
// edge, and a block of 32 hits spanning a jump gets a large box).  2D toy:
// one band; the code is a band of x over the quantised y.  Per event (one
// CTA, or one thread-block cluster for few events), in super-chunks of up to
// SUPER consecutive hits: the hits are grouped by band (stably), each band's
// run is cut into chunks of up to SORT_CAP hits, and each chunk is sorted by
// the 32-bit key (code, position in the chunk) - keys are distinct and the
// order deterministic.  A super-chunk of at most SORT_CAP hits is one chunk
// (the band is the code's top bits, so one sort already groups it).  Sorting
// a band whole, rather than cutting the event into chunks that each span all
// bands, keeps each region of a band in one run of blocks: on 16.5k-hit
// events it halves the blocks a point cannot skip.
//
// The box of a block is (umin, umax, vmin, vmax, |z|min, |z|max) for the
// slope model: since s^2 = z^2 |(u, v) - theta|^2, it bounds s^2 from below
// by |z|min^2 dist(theta, box)^2; 2D toy: (xmin, xmax, ymin, ymax, 0, 0).
// The code only orders the hits; the boxes use the exact float32 values.
// The sorted hits are written to the output in place of the event's hits
// (same CSR offsets); block b of event e (sorted hits 32b .. 32b+31) gets a
// box at index box_base(e) + b with box_base(e) = floor(offsets[e] / 32) + e,
// which never overlaps the next event's boxes.  A box holding a non-finite
// value is made infinite, so it is never skipped.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace retina {

constexpr int PREP_THREADS = 1024;
constexpr int IDX_BITS = 13;
constexpr int SORT_CAP = 1 << IDX_BITS;  // 8192 hits per sorted chunk
constexpr int SUPER = 32768;             // hits grouped by band at a time (16-bit positions)
constexpr int N_BANDS = 8;               // band values 0 .. 6 (slope model), 0 (toy)

// Shared scratch of the band grouping: positions g[SUPER] (uint16), then ints
// band starts [N_BANDS + 1], running counts [N_BANDS], tile totals [N_BANDS],
// per-warp counts [32][N_BANDS].
constexpr int GROUP_INTS = (N_BANDS + 1) + N_BANDS + N_BANDS + 32 * N_BANDS;
constexpr size_t GROUP_BYTES = (size_t)SUPER * sizeof(uint16_t) + GROUP_INTS * sizeof(int);

// v quantised on [lo, lo + 1 / inv_range] to the integers 0 .. levels
__device__ __forceinline__ uint32_t quant(float v, float lo, float inv_range, float levels) {
    float t = (v - lo) * inv_range;
    t = isfinite(t) ? fminf(fmaxf(t, 0.f), 1.f) : (t > 0.f ? 1.f : 0.f);
    return (uint32_t)(t * levels);
}

// band of a hit: slope model |z| octaves [0,16), [16,32), ..., [512, inf)
// (NaN in the last); 2D toy: 0
__device__ __forceinline__ uint32_t hit_band(const float4 h, int model) {
    if (model != RETINA_VELO_SLOPES) return 0;
    const float az = fabsf(h.z);
    uint32_t band = 0;
    for (float lim = 16.f; band < 6 && !(az < lim); lim *= 2.f) ++band;
    return band;
}

// spatial code of a hit, below 2^19, its band in the top bits (only orders
// the hits; any value is valid)
__device__ __forceinline__ uint32_t hit_code(const float4 h, int model) {
    if (model == RETINA_VELO_SLOPES) {
        const float rz = __frcp_rn(h.z);
        return (hit_band(h, model) << 16) |
               hilbert_index<8>(quant(h.x * rz, -1.f, 0.5f, 255.f), quant(h.y * rz, -1.f, 0.5f, 255.f));
    }
    return ((float_order_key(h.x) >> 25) << 7) | quant(h.y, -8.f, 1.f / 16.f, 127.f);
}

// Stable grouping of the positions 0 .. n-1 (n <= SUPER) of the hits at base
// by band: on return g[bs[q] .. bs[q+1]) lists, in increasing order, the
// positions whose hit has band q.  All threads of the CTA call it (at least
// N_BANDS warps, at most 32); it ends with a barrier.
__device__ __forceinline__ void group_by_band(const float4 *__restrict__ hits, int64_t base, int n, int model, uint16_t *g,
                              int *si) {
    int *bs = si, *run = bs + N_BANDS + 1, *tot = run + N_BANDS, *wc = tot + N_BANDS;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (tid < N_BANDS) run[tid] = 0;
    __syncthreads();
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {  // band counts
        const int i = t0 + tid;
        const int b = i < n ? (int)hit_band(__ldg(hits + base + i), model) : N_BANDS;
#pragma unroll
        for (int q = 0; q < N_BANDS; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, b == q);
            if (lane == 0 && m) atomicAdd(&run[q], __popc(m));
        }
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int q = 0; q < N_BANDS; ++q) {
            bs[q] = acc;
            acc += run[q];
            run[q] = 0;
        }
        bs[N_BANDS] = acc;
    }
    __syncthreads();
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {  // stable scatter, one tile of blockDim positions at a time
        const int i = t0 + tid;
        const int b = i < n ? (int)hit_band(__ldg(hits + base + i), model) : N_BANDS;
        int r = 0;
#pragma unroll
        for (int q = 0; q < N_BANDS; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, b == q);
            if (b == q) r = __popc(m & lt);
            if (lane == 0) wc[w * N_BANDS + q] = __popc(m);
        }
        __syncthreads();
        if (w < N_BANDS) {  // warp q: exclusive scan of band q's per-warp counts, in place
            const int c = lane < nw ? wc[lane * N_BANDS + w] : 0;
            int acc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, acc, o);
                if (lane >= o) acc += u;
            }
            if (lane < nw) wc[lane * N_BANDS + w] = acc - c;
            if (lane == 31) tot[w] = acc;
        }
        __syncthreads();
        if (b < N_BANDS) g[bs[b] + run[b] + wc[w * N_BANDS + b] + r] = (uint16_t)i;
        __syncthreads();
        if (tid < N_BANDS) run[tid] += tot[tid];
    }
    __syncthreads();
}

// One chunk: positions p0 .. p0 + n - 1 of the super-chunk at base (hit
// base + g[p] of the grouping, or base + p without one).  Keys of chunk
// positions t R + r (padding ~0 sorts last), sorted, then the hits gathered
// in key order to sorted[base + p0 ..].
template <int R>
__device__ __forceinline__ void sort_and_gather(const float4 *__restrict__ hits, int64_t base,
                                                const uint16_t *__restrict__ g, int p0, int n, int model,
                                                float4 *__restrict__ sorted, uint32_t *x) {
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        v[r] = 0xffffffffu;
        if (i < n) {
            const int src = g ? (int)g[p0 + i] : p0 + i;
            v[r] = (hit_code(__ldg(hits + base + src), model) << IDX_BITS) | (uint32_t)i;
        }
    }
    bitonic_sort_regs<uint32_t, R, PREP_THREADS>(v, x);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        if (i < n) {
            const int j = p0 + (int)(v[r] & (SORT_CAP - 1));
            sorted[base + p0 + i] = __ldg(hits + base + (g ? (int)g[j] : j));
        }
    }
}

__device__ __forceinline__ void sort_chunk(const float4 *__restrict__ hits, int64_t base, const uint16_t *g, int p0,
                                           int n, int model, float4 *__restrict__ sorted, uint32_t *x) {
    if (n <= PREP_THREADS)
        sort_and_gather<1>(hits, base, g, p0, n, model, sorted, x);
    else if (n <= 2 * PREP_THREADS)
        sort_and_gather<2>(hits, base, g, p0, n, model, sorted, x);
    else if (n <= 4 * PREP_THREADS)
        sort_and_gather<4>(hits, base, g, p0, n, model, sorted, x);
    else
        sort_and_gather<8>(hits, base, g, p0, n, model, sorted, x);
}

// Boxes of the blocks of 32 sorted hits starting at chunk positions lo .. hi
// (multiples of 32 but the chunk's last block): one warp per block, lane l
// reads hit 32 b + l, the warp reduces min / max.
__device__ __forceinline__ void chunk_boxes(const float4 *__restrict__ sorted, int64_t base, int n, int lo, int hi,
                                            int model, int64_t box0, float4 *__restrict__ boxes) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int b_lo = lo / 32, b_hi = (hi + 31) / 32;
    for (int b = b_lo + (tid >> 5); b < b_hi; b += blockDim.x / 32) {
        const int k = b * 32 + lane;
        float a = INFINITY, c = INFINITY, w = INFINITY, a2 = -INFINITY, c2 = -INFINITY, w2 = -INFINITY;
        bool finite = true;
        if (k < n) {
            const float4 h = sorted[base + k];
            if (model == RETINA_VELO_SLOPES) {
                a = h.x / h.z;  // slopes; z = 0 gives a non-finite box
                c = h.y / h.z;
                w = fabsf(h.z);
            } else {
                a = h.x;
                c = h.y;
                w = 0.f;
            }
            finite = isfinite(a) && isfinite(c) && isfinite(w);
            a2 = a;
            c2 = c;
            w2 = w;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            c = fminf(c, __shfl_xor_sync(0xffffffffu, c, o));
            w = fminf(w, __shfl_xor_sync(0xffffffffu, w, o));
            a2 = fmaxf(a2, __shfl_xor_sync(0xffffffffu, a2, o));
            c2 = fmaxf(c2, __shfl_xor_sync(0xffffffffu, c2, o));
            w2 = fmaxf(w2, __shfl_xor_sync(0xffffffffu, w2, o));
        }
        finite = __all_sync(0xffffffffu, finite);
        if (lane != 0) continue;
        float xl = a, xh = a2, yl = c, yh = c2, zl = w, zh = w2;
        if (!finite) {
            xl = yl = zl = -INFINITY;
            xh = yh = zh = INFINITY;
        }
        const int64_t bi = box0 + b;
        boxes[2 * bi] = make_float4(xl, xh, yl, yh);
        boxes[2 * bi + 1] = make_float4(zl, zh, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(PREP_THREADS)
prepare_hits_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, int model,
                    float4 *__restrict__ sorted, float4 *__restrict__ boxes) {
    extern __shared__ __align__(16) uint32_t keys[];  // [SORT_CAP], then the grouping scratch
    uint16_t *g = reinterpret_cast<uint16_t *>(keys + SORT_CAP);
    int *si = reinterpret_cast<int *>(g + SUPER);
    const int e = blockIdx.x;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    const int64_t box_base = (off[e] < 0 ? 0 : (off[e] > n_hits ? n_hits : off[e])) / 32 + e;
    for (int64_t s0 = 0; s0 < H; s0 += SUPER) {
        const int ns = (int)((H - s0) < SUPER ? (H - s0) : SUPER);
        const int64_t base = hb + s0;
        if (ns <= SORT_CAP) {
            sort_chunk(hits, base, nullptr, 0, ns, model, sorted, keys);
        } else {
            group_by_band(hits, base, ns, model, g, si);
            for (int q = 0; q < N_BANDS; ++q) {
                const int q0 = si[q], q1 = si[q + 1];
                for (int p0 = q0; p0 < q1; p0 += SORT_CAP) {
                    sort_chunk(hits, base, g, p0, (q1 - p0) < SORT_CAP ? (q1 - p0) : SORT_CAP, model, sorted, keys);
                    __syncthreads();
                }
            }
        }
        __syncthreads();  // the super-chunk's gathered hits, read back for its boxes
        chunk_boxes(sorted, base, ns, 0, ns, model, box_base + s0 / 32, boxes);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Cluster variant: CL CTAs of CL_THREADS threads per event (one thread-block
// cluster) sort each chunk of up to SORT_CAP keys together, CTA r owning chunk
// positions r P .. r P + P - 1 with P = CL_THREADS x (1, 2 or 4 keys per
// thread, the fewest that hold the chunk; shorter chunks pad with ~0 keys).
// Bitonic stages whose partner lies in another CTA read it from that CTA's
// shared memory (distributed shared memory) between cluster barriers; the
// rest is bitonic_sort_regs's in-thread / shuffle / shared exchange.  Same
// keys, same total order: the same output as prepare_hits_kernel, with CL SMs
// per event instead of one (8 CTAs of 256 threads measured fastest: 13.9 us
// per 3.9k-hit event against 15.9 us for 4 CTAs of 1024).
// ---------------------------------------------------------------------------
constexpr int CL = 8, CL_THREADS = 256;  // cluster CTAs per event and their threads

template <int R>
__device__ __forceinline__ void bitonic_cluster(uint32_t (&v)[R], uint32_t *x, int rank) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    constexpr int P = CL_THREADS * R;
    constexpr int C = CL * P;
    const int t = threadIdx.x;
    const int base = rank * P;
#pragma unroll 1
    for (int k = 2; k <= C; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j >= R; j >>= 1) {
            if (j >= P) {
#pragma unroll
                for (int r = 0; r < R; ++r) x[t * R + r] = v[r];
                cl.sync();
                const uint32_t *px = cl.map_shared_rank(x, rank ^ (j / P));
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = base + t * R + r;
                    const uint32_t b = px[t * R + r];
                    const bool keep_min = ((i & k) == 0) == (i < (i ^ j));
                    v[r] = keep_min ? (v[r] < b ? v[r] : b) : (v[r] > b ? v[r] : b);
                }
                cl.sync();
            } else if (j >= 32 * R) {
#pragma unroll
                for (int r = 0; r < R; ++r) x[t * R + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int li = t * R + r, i = base + li;
                    const uint32_t b = x[li ^ j];
                    const bool keep_min = ((i & k) == 0) == (i < (i ^ j));
                    v[r] = keep_min ? (v[r] < b ? v[r] : b) : (v[r] > b ? v[r] : b);
                }
                __syncthreads();
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = base + t * R + r;
                    const uint32_t b = __shfl_xor_sync(0xffffffffu, v[r], j / R);
                    const bool keep_min = ((i & k) == 0) == (i < (i ^ j));
                    v[r] = keep_min ? (v[r] < b ? v[r] : b) : (v[r] > b ? v[r] : b);
                }
            }
        }
#pragma unroll
        for (int j = R / 2; j >= 1; j >>= 1) {
            if (j > (k >> 1)) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r & j) continue;
                const int i = base + t * R + r;
                const uint32_t a = v[r], b = v[r | j];
                if ((a > b) == ((i & k) == 0)) {
                    v[r] = b;
                    v[r | j] = a;
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void cluster_sort_gather(const float4 *__restrict__ hits, int64_t base,
                                                    const uint16_t *__restrict__ g, int p0, int n, int model,
                                                    float4 *__restrict__ sorted, uint32_t *x, int rank) {
    constexpr int P = CL_THREADS * R;
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = rank * P + t * R + r;
        v[r] = 0xffffffffu;
        if (i < n) {
            const int src = g ? (int)g[p0 + i] : p0 + i;
            v[r] = (hit_code(__ldg(hits + base + src), model) << IDX_BITS) | (uint32_t)i;
        }
    }
    bitonic_cluster<R>(v, x, rank);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = rank * P + t * R + r;
        if (i < n) {
            const int j = p0 + (int)(v[r] & (SORT_CAP - 1));
            sorted[base + p0 + i] = __ldg(hits + base + (g ? (int)g[j] : j));
        }
    }
}

// Sorts one chunk over the cluster; returns the chunk positions per CTA.
__device__ __forceinline__ int cluster_sort_chunk(const float4 *__restrict__ hits, int64_t base, const uint16_t *g,
                                                  int p0, int n, int model, float4 *__restrict__ sorted, uint32_t *x,
                                                  int rank) {
    if (n <= CL * CL_THREADS) {
        cluster_sort_gather<1>(hits, base, g, p0, n, model, sorted, x, rank);
        return CL_THREADS;
    }
    if (n <= 2 * CL * CL_THREADS) {
        cluster_sort_gather<2>(hits, base, g, p0, n, model, sorted, x, rank);
        return 2 * CL_THREADS;
    }
    cluster_sort_gather<4>(hits, base, g, p0, n, model, sorted, x, rank);
    return 4 * CL_THREADS;
}

__global__ void __launch_bounds__(CL_THREADS, 1)
prepare_hits_cluster_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                            int model, float4 *__restrict__ sorted, float4 *__restrict__ boxes) {
    __shared__ uint32_t x[SORT_CAP / CL];
    extern __shared__ __align__(16) uint16_t g[];  // [SUPER], then the grouping's ints
    int *si = reinterpret_cast<int *>(g + SUPER);
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    pdl_release();  // the grid kernel may be scheduled once every CTA has started
    const int e = blockIdx.x / CL, rank = blockIdx.x % CL;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    const int64_t box_base = (off[e] < 0 ? 0 : (off[e] > n_hits ? n_hits : off[e])) / 32 + e;
    for (int64_t s0 = 0; s0 < H; s0 += SUPER) {
        const int ns = (int)((H - s0) < SUPER ? (H - s0) : SUPER);
        const int64_t base = hb + s0;
        // every CTA groups a super-chunk of more than SORT_CAP hits itself (the
        // same result); one of at most SORT_CAP hits is one chunk
        const bool grouped = ns > SORT_CAP;
        if (grouped) {
            group_by_band(hits, base, ns, model, g, si);
        } else {
            if (threadIdx.x <= N_BANDS) si[threadIdx.x] = threadIdx.x == 0 ? 0 : ns;
            __syncthreads();
        }
        int P = 0;
        for (int q = 0; q < N_BANDS; ++q) {
            const int q0 = si[q], q1 = si[q + 1];
            for (int p0 = q0; p0 < q1; p0 += SORT_CAP) {
                P = cluster_sort_chunk(hits, base, grouped ? g : nullptr, p0,
                                       (q1 - p0) < SORT_CAP ? (q1 - p0) : SORT_CAP, model, sorted, x, rank);
                if (grouped) cl.sync();  // x is reused by the next chunk's exchanges
            }
        }
        int lo, hi;
        if (grouped) {
            __threadfence();
            cl.sync();  // a block's hits may come from several CTAs' gathers
            const int per = (((ns + 31) / 32) + CL - 1) / CL * 32;  // positions per CTA, whole blocks
            lo = rank * per;
            hi = (rank + 1) * per < ns ? (rank + 1) * per : ns;
        } else {
            __syncthreads();  // this CTA's gathered hits, read back for its boxes
            lo = rank * P;
            hi = (rank + 1) * P < ns ? (rank + 1) * P : ns;
        }
        if (lo < ns) chunk_boxes(sorted, base, ns, lo, hi, model, box_base + s0 / 32, boxes);
        cl.sync();  // x and the grouping scratch are reused by the next super-chunk
    }
}

int64_t prepared_box_count(int64_t n_hits, int n_events) { return n_hits / 32 + n_events + 1; }

cudaError_t launch_prepare_hits(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                                float4 *sorted, float4 *boxes, cudaStream_t st) {
    // few events (latency): a cluster of CL SMs per event; batches that fill
    // the GPU many times over (throughput): one CTA per event, no cluster
    // exchanges
    if ((int64_t)n_events * CL <= 4LL * sm_count()) {
        cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(prepare_hits_cluster_kernel), GROUP_BYTES);
        if (aerr != cudaSuccess) return aerr;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(n_events * CL));
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = GROUP_BYTES;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        count_launches(1);
        return cudaLaunchKernelEx(&cfg, prepare_hits_cluster_kernel, hits, n_hits, off, model, sorted, boxes);
    }
    const size_t smem = (size_t)SORT_CAP * sizeof(uint32_t) + GROUP_BYTES;
    {
        cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(prepare_hits_kernel), smem);
        if (aerr != cudaSuccess) return aerr;
    }
    prepare_hits_kernel<<<n_events, PREP_THREADS, smem, st>>>(hits, n_hits, off, model, sorted, boxes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
