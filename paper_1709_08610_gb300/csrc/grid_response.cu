// Grid of units: R_ij = R(theta_ij) for every cell (Section 2, Eq. 2).
//
// Two kernels compute the same sum over hits:
//
// * grid_sep_kernel (slope model only).  For theta = (t_x, t_y) and a hit
//   (x, y, z) the squared distance splits into per-axis parts,
//   s^2 = (x - t_x z)^2 + (y - t_y z)^2, so each term of Eq. 1 factorises:
//   exp(-s^2/sigma^2) = exp(-(x - t_x z)^2/sigma^2) * exp(-(y - t_y z)^2/sigma^2).
//   Over an axis-aligned grid, R_ij = sum_k A_ik B_jk with
//   A_ik = exp(-(x_k - t_x,i z_k)^2/sigma^2), B_jk = exp(-(y_k - t_y,j z_k)^2/sigma^2):
//   a dense contraction over hits.  A CTA owns a 128 x 128 block of cells,
//   builds the A and B panels of a 32-hit chunk in shared memory (MUFU ex2,
//   (n0 + n1) exps per hit instead of n0 * n1), then each thread accumulates
//   an 8 x 8 outer product with FP32 FMAs (one FMA per pair).
//
// * grid_direct_kernel (both models).  Each pair (cell, hit) evaluates its
//   own exp on the MUFU pipe; per-axis parts of the distance are shared by a
//   thread's 4 x 4 cells so a pair costs one FMA, one ex2 and one add
//   (slope model) or sub, mul, mul, ex2, add (2D toy).
//
// Both kernels split an event's hits into `splits` slices (one CTA per
// (tile, slice, event)) so that a single event fills the GPU; slice partial
// grids are then summed in fixed slice order by reduce_partials_kernel, so
// results are deterministic.
#include "grid_device.cuh"

namespace retina {

constexpr int SEP_BM = 128, SEP_BN = 128, SEP_BK = 32, SEP_THREADS = 256;
constexpr int DIR_TILE = 64, DIR_THREADS = 256, DIR_CHUNK = 512;

__device__ __forceinline__ void slice_range(const int64_t *off, int64_t n_hits, int e, int s, int splits, int align,
                                            int64_t &k0, int64_t &k1) {
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t H = he - hb;
    int64_t per = (H + splits - 1) / splits;
    per = (per + align - 1) / align * align;
    k0 = hb + (int64_t)s * per;
    k1 = k0 + per < he ? k0 + per : he;
}

template <int MODEL>
__device__ __forceinline__ bool block_zero_direct(const float4 A, const float4 B, const TileRange &r, float kk) {
    if (!isfinite(B.x)) return false;
    if (MODEL == RETINA_VELO_SLOPES) {
        const float du = gap_ii(r.t0l, r.t0h, A.x, A.y), dv = gap_ii(r.t1l, r.t1h, A.z, A.w);
        return (du * du + dv * dv) * (B.x * B.x) * kk > GRID_CULL_EXPONENT;
    }
    // 2D toy, box (xmin, xmax, ymin, ymax): r = y - alpha x - beta with alpha
    // in [t0l, t0h] and beta in [t1l, t1h], by interval arithmetic
    const float p0 = r.t0l * A.x, p1 = r.t0l * A.y, p2 = r.t0h * A.x, p3 = r.t0h * A.y;
    const float pmin = fminf(fminf(p0, p1), fminf(p2, p3)), pmax = fmaxf(fmaxf(p0, p1), fmaxf(p2, p3));
    const float lo = A.z - pmax - r.t1h, hi = A.w - pmin - r.t1l;
    const float d = fmaxf(fmaxf(lo, -hi), 0.f);
    const float slack = 1e-6f * (fabsf(A.z) + fabsf(A.w) + fabsf(pmin) + fabsf(pmax) + fabsf(r.t1l) + fabsf(r.t1h));
    const float dd = fmaxf(d - slack, 0.f);
    return dd * dd * kk > GRID_CULL_EXPONENT;
}

__global__ void __launch_bounds__(SEP_THREADS, 2)
grid_sep_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                const float4 *__restrict__ boxes, GridDev g, float kk, int splits, int tiles0,
                float *__restrict__ out, int64_t split_stride, int64_t event_stride,
                unsigned long long *__restrict__ work) {
    __shared__ __align__(16) float sA[SEP_BK][SEP_BM];
    __shared__ __align__(16) float sB[SEP_BK][SEP_BN];
    __shared__ unsigned keep_mask[SEP_THREADS / 32];
    const int e = blockIdx.z, s = blockIdx.y;
    const int ti0 = (blockIdx.x % tiles0) * SEP_BM;
    const int tj0 = (blockIdx.x / tiles0) * SEP_BN;
    int64_t k0, k1;
    slice_range(off, n_hits, e, s, splits, SEP_BK, k0, k1);

    const int t = threadIdx.x;
    // panel-building role: one cell per axis, every other hit of the chunk
    const int ci = t & (SEP_BM - 1), hpar = t >> 7;
    const float t0 = cell_centre(g.lo0, g.step0, ti0 + ci);
    const float t1 = cell_centre(g.lo1, g.step1, tj0 + ci);
    // contraction role: 8 x 8 cells per thread (two 4-wide groups per axis)
    const int tm = t & 15, tn = t >> 4;

    // acc2[a][c] packs the accumulators of cells (a, 2c) and (a, 2c + 1)
    unsigned long long acc2[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[a][c] = 0ull;

    // blocks of this slice that can contribute to this tile, 256 at a time
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const float4 *gbox = boxes ? boxes + 2 * (hb / 32 + e) : nullptr;
    const TileRange tr = tile_range(g, ti0, tj0, SEP_BM, SEP_BN);
    const int64_t n_chunks = (k1 - k0 + SEP_BK - 1) / SEP_BK;
    const int64_t b_first = (k0 - hb) / SEP_BK;
    int64_t done_hits = 0;
    for (int64_t cb = 0; cb < n_chunks; cb += SEP_THREADS) {
        const int64_t c = cb + t;
        bool keep = c < n_chunks;
        if (keep && gbox) {
            const float4 A = __ldg(gbox + 2 * (b_first + c)), B = __ldg(gbox + 2 * (b_first + c) + 1);
            keep = !block_zero_sep(A, B, tr, kk);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncthreads();  // previous window's masks are no longer read
        if ((t & 31) == 0) keep_mask[t >> 5] = bal;
        __syncthreads();
        for (int w = 0; w < SEP_THREADS / 32; ++w) {
            unsigned m = keep_mask[w];
            while (m) {
                const int64_t kb = k0 + (cb + 32 * w + __ffs(m) - 1) * SEP_BK;
                m &= m - 1;
                done_hits += (k1 - kb) < SEP_BK ? (k1 - kb) : SEP_BK;
                __syncthreads();
#pragma unroll 4
                for (int mm = 0; mm < SEP_BK / 2; ++mm) {
                    const int kc = hpar + 2 * mm;
                    const int64_t k = kb + kc;
                    float va = 0.f, vb = 0.f;
                    if (k < k1) {
                        const float4 h = __ldg(hits + k);
                        const float u = __fmaf_rn(-t0, h.z, h.x);  // x - t_x z, one rounding
                        const float v = __fmaf_rn(-t1, h.z, h.y);  // y - t_y z
                        va = ex2_mufu(-(u * u) * kk);
                        vb = ex2_mufu(-(v * v) * kk);
                    }
                    sA[kc][ci] = va;
                    sB[kc][ci] = vb;
                }
                __syncthreads();
#pragma unroll
                for (int kc = 0; kc < SEP_BK; ++kc) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(&sA[kc][tm * 4]);
                    const float4 a1 = *reinterpret_cast<const float4 *>(&sA[kc][64 + tm * 4]);
                    // {b_2c, b_2c+1} pairs for the thread's 8 cells along theta1
                    const ulonglong2 b03 = *reinterpret_cast<const ulonglong2 *>(&sB[kc][tn * 4]);
                    const ulonglong2 b47 = *reinterpret_cast<const ulonglong2 *>(&sB[kc][64 + tn * 4]);
                    const float af[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const unsigned long long bv[4] = {b03.x, b03.y, b47.x, b47.y};
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const unsigned long long aa = pack2(af[a], af[a]);  // {a_i, a_i}
#pragma unroll
                        for (int c = 0; c < 4; ++c) ffma2_rn(acc2[a][c], aa, bv[c]);
                    }
                }
            }
        }
    }

    if (work && t == 0 && done_hits > 0) {
        const int64_t cw = (g.n0 - ti0 < SEP_BM ? g.n0 - ti0 : SEP_BM), ch = (g.n1 - tj0 < SEP_BN ? g.n1 - tj0 : SEP_BN);
        atomicAdd(work + RETINA_WORK_GRID, (unsigned long long)(done_hits * cw * ch));
    }
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[a][2 * c] = __uint_as_float((unsigned)(acc2[a][c] & 0xffffffffull));
            acc[a][2 * c + 1] = __uint_as_float((unsigned)(acc2[a][c] >> 32));
        }
    float *dst = out + (int64_t)s * split_stride + (int64_t)e * event_stride;
    const bool vec = (g.n0 % 4) == 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int row = tj0 + (b < 4 ? tn * 4 + b : 64 + tn * 4 + (b - 4));
        if (row >= g.n1) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int col = ti0 + half * 64 + tm * 4;
            float *p = dst + (int64_t)row * g.n0 + col;
            const float v0 = acc[half * 4 + 0][b], v1 = acc[half * 4 + 1][b];
            const float v2 = acc[half * 4 + 2][b], v3 = acc[half * 4 + 3][b];
            if (vec && col + 3 < g.n0) {
                *reinterpret_cast<float4 *>(p) = make_float4(v0, v1, v2, v3);
            } else {
                if (col + 0 < g.n0) p[0] = v0;
                if (col + 1 < g.n0) p[1] = v1;
                if (col + 2 < g.n0) p[2] = v2;
                if (col + 3 < g.n0) p[3] = v3;
            }
        }
    }
}

template <int MODEL>
__global__ void __launch_bounds__(DIR_THREADS)
grid_direct_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                   const float4 *__restrict__ boxes, GridDev g, float kk, float sk, int splits, int tiles0,
                   float *__restrict__ out, int64_t split_stride, int64_t event_stride,
                   unsigned long long *__restrict__ work) {
    __shared__ float4 sh[DIR_CHUNK];
    __shared__ int blk_list[DIR_CHUNK / 32];
    __shared__ int blk_count;
    const int e = blockIdx.z, s = blockIdx.y;
    const int ti0 = (blockIdx.x % tiles0) * DIR_TILE;
    const int tj0 = (blockIdx.x / tiles0) * DIR_TILE;
    int64_t k0, k1;
    slice_range(off, n_hits, e, s, splits, 32, k0, k1);
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const float4 *gbox = boxes ? boxes + 2 * (hb / 32 + e) : nullptr;
    const TileRange tr = tile_range(g, ti0, tj0, DIR_TILE, DIR_TILE);
    float c0[4], c1[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        c0[a] = cell_centre(g.lo0, g.step0, ti0 + tx + 16 * a);
        c1[a] = cell_centre(g.lo1, g.step1, tj0 + ty + 16 * a);
    }
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

    for (int64_t kb = k0; kb < k1; kb += DIR_CHUNK) {
        const int span = (int)((k1 - kb) < DIR_CHUNK ? (k1 - kb) : DIR_CHUNK);
        const int nb = (span + 31) / 32;
        __syncthreads();
        if (t < 32) {  // ordered list of the chunk's blocks that can contribute
            bool keep = t < nb;
            if (keep && gbox) {
                const int64_t b = (kb - hb) / 32 + t;
                keep = !block_zero_direct<MODEL>(__ldg(gbox + 2 * b), __ldg(gbox + 2 * b + 1), tr, kk);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) blk_list[__popc(bal & ((1u << t) - 1u))] = t;
            if (t == 0) blk_count = __popc(bal);
        }
        __syncthreads();
        const int nk = blk_count;
        int n = 0;
        int64_t done_hits = 0;
        for (int q = 0; q < nk; ++q) {  // gather the kept blocks' hits, in order
            const int b = blk_list[q];
            const int len = (span - 32 * b) < 32 ? (span - 32 * b) : 32;
            for (int i = t; i < len; i += DIR_THREADS) sh[n + i] = __ldg(hits + kb + 32 * b + i);
            n += len;
        }
        done_hits += n;
        if (work && t == 0 && n > 0) {
            const int64_t cw = (g.n0 - ti0 < DIR_TILE ? g.n0 - ti0 : DIR_TILE), ch = (g.n1 - tj0 < DIR_TILE ? g.n1 - tj0 : DIR_TILE);
            atomicAdd(work + RETINA_WORK_GRID, (unsigned long long)(n * cw * ch));
        }
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const float4 h = sh[i];
            if (MODEL == RETINA_VELO_SLOPES) {
                float u[4], vv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) u[a] = __fmaf_rn(-c0[a], h.z, h.x) * sk;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float v = __fmaf_rn(-c1[b], h.z, h.y) * sk;
                    vv[b] = v * v;
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] += ex2_mufu(-__fmaf_rn(u[a], u[a], vv[b]));
            } else {
                float w[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) w[a] = __fmaf_rn(-c0[a], h.x, h.y);  // y - alpha x
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float r = w[a] - c1[b];                          // minus beta
                        acc[a][b] += ex2_mufu(-(r * r) * kk);
                    }
            }
        }
    }
    float *dst = out + (int64_t)s * split_stride + (int64_t)e * event_stride;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int row = tj0 + ty + 16 * b;
        if (row >= g.n1) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int col = ti0 + tx + 16 * a;
            if (col < g.n0) dst[(int64_t)row * g.n0 + col] = acc[a][b];
        }
    }
}

// R = sum of the slice partials in slice order.  Four cells per thread (16-byte
// loads when the layout allows), the slices' loads issued eight at a time
// before their adds so that they overlap; the adds keep slice order.
__global__ void reduce_partials_kernel(const float *__restrict__ part, int splits, int64_t split_stride, int64_t n,
                                       float *__restrict__ R) {
    pdl_wait();  // launched as a dependent of the slice kernel
    const int64_t n4 = (split_stride % 4 == 0) ? n / 4 : 0;
    const float4 *p4 = reinterpret_cast<const float4 *>(part);
    const int64_t st4 = split_stride / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int s0 = 0; s0 < splits; s0 += 8) {
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (s0 + u < splits) x[u] = __ldg(p4 + (int64_t)(s0 + u) * st4 + i);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (s0 + u < splits) {
                    v.x += x[u].x;
                    v.y += x[u].y;
                    v.z += x[u].z;
                    v.w += x[u].w;
                }
        }
        reinterpret_cast<float4 *>(R)[i] = v;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int s = 0; s < splits; ++s) v += part[(int64_t)s * split_stride + i];
        R[i] = v;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

GridPlan plan_grid(int n_events, int model, const retina_grid *g, int flags, int forced_splits) {
    GridPlan p;
    p.separable = (model == RETINA_VELO_SLOPES) && (flags != RETINA_GRID_DIRECT);
    p.tc = p.separable && (flags == RETINA_GRID_TENSOR ||
                           (flags == RETINA_GRID_AUTO && option_value(RETINA_OPT_GRID_TC) != 0));
    const int tile = p.separable ? SEP_BM : DIR_TILE;
    p.tiles0 = (g->n[0] + tile - 1) / tile;
    p.tiles1 = (g->n[1] + tile - 1) / tile;
    // tensor cores: 128 x 256 tiles (two CTAs per SM, a quarter less
    // shared-memory traffic per multiply-add) when the 128 x 128 tiles would
    // fill the GPU eight times over, else 128 x 128 (three CTAs per SM, more
    // CTAs for few events)
    p.tc_bn = 128;
    if (p.tc && (int64_t)p.tiles0 * p.tiles1 * (n_events > 0 ? n_events : 1) >= 8LL * sm_count()) {
        p.tc_bn = 256;
        p.tiles1 = (g->n[1] + 255) / 256;
    }
    const int64_t ctas = (int64_t)p.tiles0 * p.tiles1 * (n_events > 0 ? n_events : 1);
    const int per_sm = p.tc ? (p.tc_bn == 256 ? 2 : 3) : (p.separable ? 2 : 4);
    const int64_t target = 4LL * sm_count() * per_sm;
    int64_t s = (target + ctas - 1) / ctas;
    if (s < 1) s = 1;
    if (s > 32) s = 32;
    p.splits = forced_splits > 0 ? forced_splits : (int)s;
    return p;
}

size_t grid_partials_bytes(const GridPlan &p, int n_events, const retina_grid *g) {
    if (p.splits <= 1) return 0;
    return (size_t)p.splits * (size_t)n_events * (size_t)g->n[0] * (size_t)g->n[1] * sizeof(float);
}

cudaError_t launch_grid_response(const GridPlan &p, const float4 *hits, int64_t n_hits, const int64_t *off,
                                 const float4 *boxes, int n_events, int model,
                                 const retina_grid *g, float sigma, float *R, float *partials, cudaStream_t st) {
    GridDev gd{g->lo[0], g->lo[1], g->step[0], g->step[1], g->n[0], g->n[1]};
    const double kkd = kLog2e / ((double)sigma * (double)sigma);
    const float kk = (float)kkd;
    const float sk = (float)sqrt(kkd);
    const int64_t cells = (int64_t)g->n[0] * g->n[1];
    float *dst = p.splits > 1 ? partials : R;
    const int64_t split_stride = cells * n_events;
    dim3 grid(p.tiles0 * p.tiles1, p.splits, n_events);
    if (p.tc) {
        int32_t *flag = device_error_flag();
        if (!flag) return cudaErrorInvalidSymbol;
        cudaError_t lerr = launch_grid_tc(p.tc_bn, grid, st, hits, n_hits, off, boxes, gd, kk, p.splits, p.tiles0, dst,
                                          split_stride, cells, flag);
        if (lerr != cudaSuccess) return lerr;
    } else if (p.separable) {
        grid_sep_kernel<<<grid, SEP_THREADS, 0, st>>>(hits, n_hits, off, boxes, gd, kk, p.splits, p.tiles0, dst, split_stride, cells,
                                                      work_counters());
    } else if (model == RETINA_VELO_SLOPES) {
        grid_direct_kernel<RETINA_VELO_SLOPES>
            <<<grid, DIR_THREADS, 0, st>>>(hits, n_hits, off, boxes, gd, kk, sk, p.splits, p.tiles0, dst, split_stride,
                                                        cells, work_counters());
    } else {
        grid_direct_kernel<RETINA_TOY2D>
            <<<grid, DIR_THREADS, 0, st>>>(hits, n_hits, off, boxes, gd, kk, sk, p.splits, p.tiles0, dst, split_stride,
                                                        cells, work_counters());
    }
    count_launches(1);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (p.splits > 1) {
        count_launches(1);
        const int64_t n = split_stride;
        int blocks = (int)((n / 4 + 255) / 256);
        const int cap = sm_count() * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        PrioLaunch L(dim3(blocks), dim3(256), 0, st, true);
        err = cudaLaunchKernelEx(&L.cfg, reduce_partials_kernel, (const float *)partials, p.splits, split_stride, n, R);
        if (err == cudaSuccess) err = cudaGetLastError();
    }
    return err;
}

}  // namespace retina
