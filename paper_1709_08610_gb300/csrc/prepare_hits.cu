// Spatial ordering of each event's hits plus a bounding box per block of 32,
// so that the response kernels can skip, exactly, blocks whose every term of
// Eq. 1 is zero in float32.
//
// Each hit gets a spatial code.  Slope model: a band of |z| (octaves from 16
// mm; 7 bands) over the index of the hit's slopes (u, v) = (x/z, y/z),
// quantised to 256 levels on [-1, 1] (clamped at the edges), along the
// Hilbert curve of order 8, whose consecutive cells always touch (a Morton
// order jumps at every quadrant edge, and a block of 32 hits spanning a jump
// gets a large box).  2D toy: a band of x over the quantised y.  Per event
// (one CTA, or one thread-block cluster for few events), each super-chunk of
// up to SUPER consecutive hits is sorted by (code, index): chunks of up to
// SORT_CAP hits are sorted by the 32-bit key (code, position in the chunk),
// then merged by rank - an element's output position is its rank in its own
// chunk plus, in every other chunk, the number of codes below its own (or
// not above it, for the chunks before its own, so that equal codes keep
// index order).  Sorting the event whole, rather than chunk by chunk, keeps
// each region of a band in one run of blocks: on 16.5k-hit events it halves
// the blocks a point cannot skip.
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
constexpr int SUPER_CHUNKS = 4;
constexpr int SUPER = SUPER_CHUNKS * SORT_CAP;  // 32768 hits sorted together

// v quantised on [lo, lo + 1 / inv_range] to the integers 0 .. levels, every
// operation rounded on its own (no multiply-add contraction with the
// caller's product), so that the documented order can be restated exactly
__device__ __forceinline__ uint32_t quant(float v, float lo, float inv_range, float levels) {
    float t = __fmul_rn(__fsub_rn(v, lo), inv_range);
    t = isfinite(t) ? fminf(fmaxf(t, 0.f), 1.f) : (t > 0.f ? 1.f : 0.f);
    return (uint32_t)__fmul_rn(t, levels);
}

// spatial code of a hit, below 2^19 (only orders the hits; any value is valid)
__device__ __forceinline__ uint32_t hit_code(const float4 h, int model) {
    if (model == RETINA_VELO_SLOPES) {
        const float az = fabsf(h.z);
        uint32_t band = 0;  // |z| octaves: [0,16), [16,32), ..., [512, inf) (NaN in the last)
        for (float lim = 16.f; band < 6 && !(az < lim); lim *= 2.f) ++band;
        const float rz = __frcp_rn(h.z);
        return (band << 16) | hilbert_index<8>(quant(__fmul_rn(h.x, rz), -1.f, 0.5f, 255.f),
                                               quant(__fmul_rn(h.y, rz), -1.f, 0.5f, 255.f));
    }
    return ((float_order_key(h.x) >> 25) << 7) | quant(h.y, -8.f, 1.f / 16.f, 127.f);
}

// key of chunk position i (n valid; padding ~0 sorts last)
__device__ __forceinline__ uint32_t chunk_key(const float4 *__restrict__ hits, int64_t base, int i, int n, int model) {
    return i < n ? ((hit_code(__ldg(hits + base + i), model) << IDX_BITS) | (uint32_t)i) : 0xffffffffu;
}

// Stable LSD radix sort of the 1024 R keys a CTA holds blocked (thread t
// holds positions t R .. t R + R - 1) by their code bits (above the
// IDX_BITS position bits), RADIX_BITS a pass.  A pass counts every thread's
// keys per digit into digit-major, thread-minor counters, scans them in
// that order, and moves each key to its digit's start plus the keys of
// that digit in earlier threads and earlier in its own thread: equal
// digits keep their order, so after the last pass the keys are in their
// one sorted order (the positions make them distinct).  Linear in the keys,
// where the bitonic network does log^2 stages of compare-exchanges.
// x: 1024 R keys of exchange; ctr: RADIX x PREP_THREADS counters.
constexpr int RADIX_BITS = 4, RADIX = 1 << RADIX_BITS;
constexpr int CODE_BITS = 32 - IDX_BITS;  // codes are below 2^19 = 2^CODE_BITS
template <int R>
__device__ __forceinline__ void radix_sort_regs(uint32_t (&v)[R], uint32_t *x, uint32_t *ctr) {
    __shared__ uint32_t wsum[PREP_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll 1
    for (int s = IDX_BITS; s < IDX_BITS + CODE_BITS; s += RADIX_BITS) {
        uint32_t off[R];
        int dg[R];
#pragma unroll
        for (int d = 0; d < RADIX; ++d) ctr[d * PREP_THREADS + t] = 0;  // this thread's column
#pragma unroll
        for (int r = 0; r < R; ++r) {
            dg[r] = (int)((v[r] >> s) & (RADIX - 1));
            off[r] = ctr[dg[r] * PREP_THREADS + t];
            ctr[dg[r] * PREP_THREADS + t] = off[r] + 1;
        }
        __syncthreads();
        // exclusive scan of the RADIX x PREP_THREADS counters in index order:
        // thread t owns entries RADIX t .. RADIX t + RADIX - 1
        uint32_t loc[RADIX], tot = 0;
#pragma unroll
        for (int j = 0; j < RADIX; ++j) {
            loc[j] = ctr[RADIX * t + j];
            tot += loc[j];
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t run = inc - tot;
        for (int i = 0; i < w; ++i) run += wsum[i];
#pragma unroll
        for (int j = 0; j < RADIX; ++j) {
            ctr[RADIX * t + j] = run;
            run += loc[j];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) x[ctr[dg[r] * PREP_THREADS + t] + off[r]] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[t * R + r];
        // the next pass first rewrites only this thread's counter column and
        // this thread's exchange reads are its own; its scatter comes after
        // two more barriers
    }
}

// Keys of chunk positions t R + r, sorted, then the hits gathered in key
// order to sorted[base ..] (a super-chunk that is one chunk).
template <int R>
__device__ __forceinline__ void sort_and_gather(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                                float4 *__restrict__ sorted, uint32_t *x, uint32_t *ctr) {
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = chunk_key(hits, base, t * R + r, n, model);
    radix_sort_regs<R>(v, x, ctr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t * R + r;
        if (i < n) sorted[base + i] = __ldg(hits + base + (int)(v[r] & (SORT_CAP - 1)));
    }
}

// The same sort, the sorted keys left in K[0 .. 1024 R) (K is also the
// sort's exchange buffer).
template <int R>
__device__ __forceinline__ void sort_keys(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                          uint32_t *K, uint32_t *ctr) {
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = chunk_key(hits, base, t * R + r, n, model);
    radix_sort_regs<R>(v, K, ctr);
    __syncthreads();  // every exchange read is done before K holds the result
#pragma unroll
    for (int r = 0; r < R; ++r) K[t * R + r] = v[r];
}

template <bool GATHER>
__device__ __forceinline__ void sort_chunk(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                           float4 *__restrict__ sorted, uint32_t *x, uint32_t *ctr) {
    if (n <= PREP_THREADS) {
        if (GATHER) sort_and_gather<1>(hits, base, n, model, sorted, x, ctr);
        else sort_keys<1>(hits, base, n, model, x, ctr);
    } else if (n <= 2 * PREP_THREADS) {
        if (GATHER) sort_and_gather<2>(hits, base, n, model, sorted, x, ctr);
        else sort_keys<2>(hits, base, n, model, x, ctr);
    } else if (n <= 4 * PREP_THREADS) {
        if (GATHER) sort_and_gather<4>(hits, base, n, model, sorted, x, ctr);
        else sort_keys<4>(hits, base, n, model, x, ctr);
    } else {
        if (GATHER) sort_and_gather<8>(hits, base, n, model, sorted, x, ctr);
        else sort_keys<8>(hits, base, n, model, x, ctr);
    }
}

// Number of the first n entries of the ascending array at(.) below thr
// (binary search; at(j) reads entry j).
template <typename At>
__device__ __forceinline__ int count_below(At &&at, int n, uint64_t thr) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)at(mid) < thr)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Keys below this bound in another chunk go before a key of code `code`:
// codes below it, and equal codes too when that chunk comes first (equal
// codes keep index order).
__device__ __forceinline__ uint64_t rank_bound(uint32_t code, bool earlier_chunk) {
    return (uint64_t)(code + (earlier_chunk ? 1u : 0u)) << IDX_BITS;
}

// size of chunk c of a super-chunk of ns hits
__device__ __forceinline__ int chunk_size(int ns, int c) {
    return ns - c * SORT_CAP < SORT_CAP ? ns - c * SORT_CAP : SORT_CAP;
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
    extern __shared__ __align__(16) uint32_t K[];  // [SUPER]: each chunk's sorted keys, then the radix counters
    uint32_t *ctr = K + SUPER;
    const int e = blockIdx.x;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    const int64_t box_base = (off[e] < 0 ? 0 : (off[e] > n_hits ? n_hits : off[e])) / 32 + e;
    for (int64_t s0 = 0; s0 < H; s0 += SUPER) {
        const int ns = (int)((H - s0) < SUPER ? (H - s0) : SUPER);
        const int64_t base = hb + s0;
        if (ns <= SORT_CAP) {
            sort_chunk<true>(hits, base, ns, model, sorted, K, ctr);
        } else {
            const int nch = (ns + SORT_CAP - 1) / SORT_CAP;
            for (int c = 0; c < nch; ++c)
                sort_chunk<false>(hits, base + c * SORT_CAP, chunk_size(ns, c), model, sorted, K + c * SORT_CAP, ctr);
            __syncthreads();
            // merge by rank: chunk c's j-th key goes to j + (keys before it in the other chunks)
            for (int c = 0; c < nch; ++c) {
                const int n = chunk_size(ns, c);
                for (int j = threadIdx.x; j < n; j += PREP_THREADS) {
                    const uint32_t key = K[c * SORT_CAP + j];
                    const uint32_t code = key >> IDX_BITS;
                    int out = j;
                    for (int c2 = 0; c2 < nch; ++c2) {
                        if (c2 == c) continue;
                        const uint32_t *K2 = K + c2 * SORT_CAP;
                        out += count_below([&](int m) { return K2[m]; }, chunk_size(ns, c2), rank_bound(code, c2 < c));
                    }
                    sorted[base + out] = __ldg(hits + base + c * SORT_CAP + (int)(key & (SORT_CAP - 1)));
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

// One chunk over the cluster: keys sorted, then either the hits gathered in
// key order (GATHER: a super-chunk that is one chunk) or this CTA's slice of
// the sorted keys kept in Ks[0 .. P).
template <int R, bool GATHER>
__device__ __forceinline__ void cluster_sort(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                             float4 *__restrict__ sorted, uint32_t *x, uint32_t *Ks, int rank) {
    constexpr int P = CL_THREADS * R;
    uint32_t v[R];
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = chunk_key(hits, base, rank * P + t * R + r, n, model);
    bitonic_cluster<R>(v, x, rank);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = rank * P + t * R + r;
        if (GATHER) {
            if (i < n) sorted[base + i] = __ldg(hits + base + (int)(v[r] & (SORT_CAP - 1)));
        } else {
            Ks[t * R + r] = v[r];
        }
    }
}

// Sorts one chunk over the cluster; returns the chunk positions per CTA.
template <bool GATHER>
__device__ __forceinline__ int cluster_sort_chunk(const float4 *__restrict__ hits, int64_t base, int n, int model,
                                                  float4 *__restrict__ sorted, uint32_t *x, uint32_t *Ks, int rank) {
    if (n <= CL * CL_THREADS) {
        cluster_sort<1, GATHER>(hits, base, n, model, sorted, x, Ks, rank);
        return CL_THREADS;
    }
    if (n <= 2 * CL * CL_THREADS) {
        cluster_sort<2, GATHER>(hits, base, n, model, sorted, x, Ks, rank);
        return 2 * CL_THREADS;
    }
    cluster_sort<4, GATHER>(hits, base, n, model, sorted, x, Ks, rank);
    return 4 * CL_THREADS;
}

__global__ void __launch_bounds__(CL_THREADS, 1)
prepare_hits_cluster_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                            int model, float4 *__restrict__ sorted, float4 *__restrict__ boxes) {
    __shared__ uint32_t x[SORT_CAP / CL];
    __shared__ uint32_t Ks[SUPER_CHUNKS][SORT_CAP / CL];  // this CTA's slice of each chunk's sorted keys
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
        int lo, hi;
        if (ns <= SORT_CAP) {
            const int P = cluster_sort_chunk<true>(hits, base, ns, model, sorted, x, nullptr, rank);
            __syncthreads();  // this CTA's gathered hits, read back for its boxes
            lo = rank * P;
            hi = (rank + 1) * P < ns ? (rank + 1) * P : ns;
        } else {
            const int nch = (ns + SORT_CAP - 1) / SORT_CAP;
            int Pc[SUPER_CHUNKS];
#pragma unroll
            for (int c = 0; c < SUPER_CHUNKS; ++c) {
                if (c >= nch) break;
                Pc[c] = cluster_sort_chunk<false>(hits, base + c * SORT_CAP, chunk_size(ns, c), model, sorted, x,
                                                  Ks[c], rank);
                cl.sync();  // x is reused by the next chunk's exchanges; every slice is stored
            }
            // merge by rank: each CTA places its own slices' keys, searching
            // the other chunks through distributed shared memory
#pragma unroll
            for (int c = 0; c < SUPER_CHUNKS; ++c) {
                if (c >= nch) break;
                const int n = chunk_size(ns, c);
                for (int m = threadIdx.x; m < Pc[c]; m += CL_THREADS) {
                    const int j = rank * Pc[c] + m;
                    if (j >= n) break;
                    const uint32_t key = Ks[c][m];
                    const uint32_t code = key >> IDX_BITS;
                    int out = j;
#pragma unroll
                    for (int c2 = 0; c2 < SUPER_CHUNKS; ++c2) {
                        if (c2 >= nch || c2 == c) continue;
                        const int P2 = Pc[c2];
                        out += count_below([&](int q) { return cl.map_shared_rank(&Ks[c2][0], q / P2)[q % P2]; },
                                           chunk_size(ns, c2), rank_bound(code, c2 < c));
                    }
                    sorted[base + out] = __ldg(hits + base + c * SORT_CAP + (int)(key & (SORT_CAP - 1)));
                }
            }
            __threadfence();
            cl.sync();  // a block's hits come from several CTAs' writes
            const int per = (((ns + 31) / 32) + CL - 1) / CL * 32;  // positions per CTA, whole blocks
            lo = rank * per;
            hi = (rank + 1) * per < ns ? (rank + 1) * per : ns;
        }
        if (lo < ns) chunk_boxes(sorted, base, ns, lo, hi, model, box_base + s0 / 32, boxes);
        cl.sync();  // x and Ks are reused (and read remotely) until every CTA is here
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
    const size_t smem = (size_t)(SUPER + RADIX * PREP_THREADS) * sizeof(uint32_t);
    {
        cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(prepare_hits_kernel), smem);
        if (aerr != cudaSuccess) return aerr;
    }
    prepare_hits_kernel<<<n_events, PREP_THREADS, smem, st>>>(hits, n_hits, off, model, sorted, boxes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
