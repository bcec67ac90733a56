// Spatial ordering of each event's hits plus a bounding box per block of 32,
// so that the response kernels can skip, exactly, blocks whose every term of
// Eq. 1 is zero in float32.
//
// Per event (one CTA, chunks of up to SORT_CAP hits): each hit gets a 32-bit
// key - a spatial code of up to 19 bits above its 13-bit index in the chunk,
// so keys are distinct and the order is deterministic - and the chunk is
// sorted by key.  Slope model: the code is a band of |z| (octaves from 16 mm)
// over a 16-bit Morton code of the hit's slopes (u, v) = (x/z, y/z)
// quantised on [-1, 1] (slopes beyond are clamped to the edges),
// and the box of a block is (umin, umax, vmin, vmax, |z|min, |z|max): since
// s^2 = z^2 |(u, v) - theta|^2, it bounds s^2 from below by
// |z|min^2 dist(theta, box)^2.  2D toy: the code is a band of x over the
// quantised y, and the box is (xmin, xmax, ymin, ymax, 0, 0).  The code only
// orders the hits; the boxes use the exact float32 values.
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
constexpr int SORT_CAP = 1 << IDX_BITS;  // 8192 hits per chunk

// Spread the 8 low bits of v to the even bit positions 0, 2, ..., 14.
__device__ __forceinline__ uint32_t spread8(uint32_t v) {
    v &= 0xffu;
    v = (v | (v << 4)) & 0x0f0fu;
    v = (v | (v << 2)) & 0x3333u;
    v = (v | (v << 1)) & 0x5555u;
    return v;
}

// v quantised on [lo, lo + 1 / inv_range] to the integers 0 .. levels
__device__ __forceinline__ uint32_t quant(float v, float lo, float inv_range, float levels) {
    float t = (v - lo) * inv_range;
    t = isfinite(t) ? fminf(fmaxf(t, 0.f), 1.f) : (t > 0.f ? 1.f : 0.f);
    return (uint32_t)(t * levels);
}

// spatial code of a hit, below 2^19 (only orders the hits; any value is valid)
__device__ __forceinline__ uint32_t hit_code(const float4 h, int model) {
    if (model == RETINA_VELO_SLOPES) {
        const float az = fabsf(h.z);
        uint32_t band = 0;  // |z| octaves: [0,16), [16,32), ..., [512, inf)
        for (float lim = 16.f; band < 6 && !(az < lim); lim *= 2.f) ++band;
        const float rz = __frcp_rn(h.z);
        const uint32_t m = spread8(quant(h.x * rz, -1.f, 0.5f, 255.f)) | (spread8(quant(h.y * rz, -1.f, 0.5f, 255.f)) << 1);
        return (band << 16) | m;
    }
    return ((float_order_key(h.x) >> 25) << 7) | quant(h.y, -8.f, 1.f / 16.f, 127.f);
}

// Keys of chunk positions t R + r (padding ~0 sorts last), sorted, then the
// hits gathered in key order.
template <int R>
__device__ __forceinline__ void sort_and_gather(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                                float4 *__restrict__ sorted, uint32_t *x) {
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        v[r] = i < n ? ((hit_code(__ldg(hits + base + i), model) << IDX_BITS) | (uint32_t)i) : 0xffffffffu;
    }
    bitonic_sort_regs<uint32_t, R, PREP_THREADS>(v, x);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        if (i < n) sorted[base + i] = __ldg(hits + base + (int)(v[r] & (SORT_CAP - 1)));
    }
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
    extern __shared__ uint32_t keys[];
    const int e = blockIdx.x;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    const int64_t box_base = (off[e] < 0 ? 0 : (off[e] > n_hits ? n_hits : off[e])) / 32 + e;
    for (int64_t c0 = 0; c0 < H; c0 += SORT_CAP) {
        const int n = (int)((H - c0) < SORT_CAP ? (H - c0) : SORT_CAP);
        const int64_t base = hb + c0;
        if (n <= PREP_THREADS)
            sort_and_gather<1>(hits, base, n, model, sorted, keys);
        else if (n <= 2 * PREP_THREADS)
            sort_and_gather<2>(hits, base, n, model, sorted, keys);
        else if (n <= 4 * PREP_THREADS)
            sort_and_gather<4>(hits, base, n, model, sorted, keys);
        else
            sort_and_gather<8>(hits, base, n, model, sorted, keys);
        __syncthreads();
        chunk_boxes(sorted, hb + c0, n, 0, n, model, box_base + c0 / 32, boxes);
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
__device__ __forceinline__ void cluster_sort_gather(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                                    float4 *__restrict__ sorted, uint32_t *x, int rank) {
    constexpr int P = CL_THREADS * R;
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = rank * P + t * R + r;
        v[r] = i < n ? ((hit_code(__ldg(hits + base + i), model) << IDX_BITS) | (uint32_t)i) : 0xffffffffu;
    }
    bitonic_cluster<R>(v, x, rank);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = rank * P + t * R + r;
        if (i < n) sorted[base + i] = __ldg(hits + base + (int)(v[r] & (SORT_CAP - 1)));
    }
}

__global__ void __launch_bounds__(CL_THREADS)
prepare_hits_cluster_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                            int model, float4 *__restrict__ sorted, float4 *__restrict__ boxes) {
    __shared__ uint32_t x[SORT_CAP / CL];
    pdl_release();  // the grid kernel may be scheduled once every CTA has started
    const int e = blockIdx.x / CL, rank = blockIdx.x % CL;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    const int64_t box_base = (off[e] < 0 ? 0 : (off[e] > n_hits ? n_hits : off[e])) / 32 + e;
    for (int64_t c0 = 0; c0 < H; c0 += SORT_CAP) {
        const int n = (int)((H - c0) < SORT_CAP ? (H - c0) : SORT_CAP);
        const int64_t base = hb + c0;
        int P;  // chunk positions per CTA: CL_THREADS x (keys per thread)
        if (n <= CL * CL_THREADS) {
            cluster_sort_gather<1>(hits, base, n, model, sorted, x, rank);
            P = CL_THREADS;
        } else if (n <= 2 * CL * CL_THREADS) {
            cluster_sort_gather<2>(hits, base, n, model, sorted, x, rank);
            P = 2 * CL_THREADS;
        } else {
            cluster_sort_gather<4>(hits, base, n, model, sorted, x, rank);
            P = 4 * CL_THREADS;
        }
        __syncthreads();  // this CTA's gathered hits, read back for its boxes
        const int lo = rank * P, hi = (rank + 1) * P < n ? (rank + 1) * P : n;
        if (lo < n) chunk_boxes(sorted, base, n, lo, hi, model, box_base + c0 / 32, boxes);
        cooperative_groups::this_cluster().sync();  // x is reused by the next chunk's exchanges
    }
}

int64_t prepared_box_count(int64_t n_hits, int n_events) { return n_hits / 32 + n_events + 1; }

cudaError_t launch_prepare_hits(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                                float4 *sorted, float4 *boxes, cudaStream_t st) {
    // few events (latency): a cluster of CL SMs per event; batches that fill
    // the GPU many times over (throughput): one CTA per event, no cluster
    // exchanges
    if ((int64_t)n_events * CL <= 4LL * sm_count()) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(n_events * CL));
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = 0;
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
    const size_t smem = (size_t)SORT_CAP * sizeof(uint32_t);
    {
        cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(prepare_hits_kernel), smem);
        if (aerr != cudaSuccess) return aerr;
    }
    prepare_hits_kernel<<<n_events, PREP_THREADS, smem, st>>>(hits, n_hits, off, model, sorted, boxes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
