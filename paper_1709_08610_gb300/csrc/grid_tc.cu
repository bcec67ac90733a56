// Grid response of the slope model (Eq. 2) as a tensor-core contraction
// (tcgen05, kind::tf32, sm_103a).
//
// For an axis-aligned (t_x, t_y) grid, exp(-s^2/sigma^2) factorises:
//   R[j][i] = sum_k A[i][k] B[j][k],  A[i][k] = ex2(-(x_k - t_x,i z_k)^2 kk),
//                                      B[j][k] = ex2(-(y_k - t_y,j z_k)^2 kk)
// (the same exponentials, formed the same way, as grid_sep_kernel).  A CTA owns
// a 128 x 256 tile of cells (128 theta_0 cells, 256 theta_1 cells); for every
// 32-hit block that can contribute to the tile (exact block skipping, as
// grid_sep_kernel) it builds the 128 x 32 and 256 x 32 FP32 panels and
// accumulates A B^T into a 128 x 256 FP32 accumulator in tensor memory with
// TF32 MMAs (M = 128, N = 256, K = 8).  The wide tile halves the A panels
// built per cell and cuts the shared-memory traffic per multiply-add (panel
// stores and the MMAs' operand reads, which share the shared-memory
// bandwidth with the panel builds) by a quarter against a 128 x 128 tile.  TF32 keeps 10 mantissa
// bits, so each panel is split into hi = (value with its 13 low mantissa bits
// cleared) and lo = value - hi (exact), and three products hi.hi + hi.lo +
// lo.hi are accumulated: every product is then within ~2^-19 of the FP32
// product, and since all terms are positive R keeps that relative accuracy.
// One thread issues the MMAs and commits them to an mbarrier; waits are
// bounded (expiry sets the library's device error flag).
#include "grid_device.cuh"

namespace retina {

namespace {

constexpr int GT_BM = 128, GT_BK = 32, GT_THREADS = 256;
constexpr int PANEL_A = GT_BM * GT_BK * 4;       // 16 KB

// shared-memory layout for tiles of BN (128 or 256) theta_1 cells: the A and
// B panels (hi, lo), the current block's 32 hits (float4), the keep masks of
// the current window (8 x u32), the mbarrier (8 B) and the TMEM address
template <int BN>
struct GtLayout {
    static constexpr int PANEL_B = BN * GT_BK * 4;
    static constexpr int OFF_AHI = 0, OFF_ALO = PANEL_A, OFF_BHI = 2 * PANEL_A, OFF_BLO = 2 * PANEL_A + PANEL_B;
    static constexpr int OFF_HITS = 2 * PANEL_A + 2 * PANEL_B;
    static constexpr int OFF_MASK = OFF_HITS + GT_BK * 16;
    static constexpr int OFF_BAR = OFF_MASK + 32;
    static constexpr int SMEM = OFF_BAR + 16;
    // kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (format 2 at bits 7-9
    // and 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
    static constexpr uint32_t IDESC =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
};
constexpr uint32_t GT_WAIT_LIMIT = 1u << 24;


__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// no-swizzle K-major descriptor; core matrices 8 rows x 16 bytes
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// byte offset of element (row m, hit k) of a 128 (or 256) x 32 FP32 K-major panel:
// core matrix (m / 8, k / 4) at (m / 8) * 1024 + (k / 4) * 128
__device__ __forceinline__ int panel_off(int m, int k) { return (m >> 3) * 1024 + (k >> 2) * 128 + (m & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    lo = v - hi;  // exact: v and hi share sign and exponent
}

__device__ __forceinline__ bool gt_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool gt_wait(uint32_t addr, uint32_t parity) {
    for (uint32_t i = 0; i < GT_WAIT_LIMIT; ++i)
        if (gt_try_wait(addr, parity)) return true;
    return false;
}

__device__ __forceinline__ void gt_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void gt_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// Grid over (tiles, hit slices, events) and partial layout as grid_sep_kernel;
// the slices interleave 32-hit blocks instead of cutting contiguous ranges.
// BN: the tile's theta_1 cells (128: three CTAs per SM; 256: two).
template <int BN>
__global__ void __launch_bounds__(GT_THREADS, 1)
grid_tc_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
               const float4 *__restrict__ boxes, GridDev g, float kk, int splits, int tiles0, float *__restrict__ out,
               int64_t split_stride, int64_t event_stride, unsigned long long *__restrict__ work,
               int32_t *__restrict__ err) {
    using L = GtLayout<BN>;
    constexpr int GT_BN = BN, GT_NCOLS = BN, NB = BN / 64;  // B rows per thread
    constexpr int OFF_AHI = L::OFF_AHI, OFF_ALO = L::OFF_ALO, OFF_BHI = L::OFF_BHI, OFF_BLO = L::OFF_BLO;
    constexpr int OFF_HITS = L::OFF_HITS, OFF_MASK = L::OFF_MASK, OFF_BAR = L::OFF_BAR;
    extern __shared__ __align__(1024) unsigned char gsm[];
    pdl_release();  // the slice reduction may be scheduled once every CTA has started
    pdl_wait();     // may be launched while the hit ordering finishes
    unsigned *keep_mask = reinterpret_cast<unsigned *>(gsm + OFF_MASK);
    uint64_t *bar = reinterpret_cast<uint64_t *>(gsm + OFF_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gsm + OFF_BAR + 8);
    const uint32_t bar_addr = smem_addr(bar);
    const int e = blockIdx.z, s = blockIdx.y;
    const int ti0 = (blockIdx.x % tiles0) * GT_BM;
    const int tj0 = (blockIdx.x / tiles0) * GT_BN;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(GT_NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_addr), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // panel role: lane l of warp w owns A rows (theta_0 cells) m = 8 (2w + a)
    // + l / 4 (a = 0, 1), B rows (theta_1 cells) m + 128 c (c < BN / 128),
    // and hits k = 4 j + l % 4 (j = 0..7), so the 32 lanes of every store hit
    // 32 different banks of the core-matrix layout
    const int lm = lane >> 2, lk = lane & 3;
    const int m0 = 16 * warp + lm, m1 = m0 + 8;
    const float t0a = cell_centre(g.lo0, g.step0, ti0 + m0), t0b = cell_centre(g.lo0, g.step0, ti0 + m1);
    int mb[NB];
    float t1[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        mb[c] = m0 + 8 * (c & 1) + 128 * (c >> 1);
        t1[c] = cell_centre(g.lo1, g.step1, tj0 + mb[c]);
    }

    // slice s takes the event's 32-hit blocks s, s + splits, s + 2 splits, ...:
    // the blocks a tile keeps cluster in the hits' spatial order, and
    // interleaving spreads them evenly over the tile's slices
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int64_t nblk = (he - hb + GT_BK - 1) / GT_BK;
    const float4 *gbox = boxes ? boxes + 2 * (hb / 32 + e) : nullptr;
    const TileRange tr = tile_range(g, ti0, tj0, GT_BM, GT_BN);
    const int64_t n_chunks = nblk > s ? (nblk - s + splits - 1) / splits : 0;
    auto block_of = [&](int64_t c) -> int64_t { return (int64_t)s + c * splits; };
    int64_t done_hits = 0;
    uint32_t phase = 0;
    bool any = false, failed = false;
    for (int64_t cb = 0; cb < n_chunks && !failed; cb += GT_THREADS) {
        const int64_t c = cb + t;
        bool keep = c < n_chunks;
        if (keep && gbox) {
            const float4 A = __ldg(gbox + 2 * block_of(c)), B = __ldg(gbox + 2 * block_of(c) + 1);
            keep = !block_zero_sep(A, B, tr, kk);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncthreads();  // previous window's masks are no longer read
        if (lane == 0) keep_mask[warp] = bal;
        __syncthreads();
        // kept blocks of the window in order; block `nxt`'s hits are loaded into
        // registers while the current block's MMAs run
        auto next_kept = [&](int after) -> int {  // first kept block index > after, or -1
            for (int w = (after + 1) >> 5; w < GT_THREADS / 32; ++w) {
                const int bit = (after + 1) - 32 * w;
                const unsigned mw = keep_mask[w] & (bit > 0 ? (~0u << bit) : ~0u);
                if (mw) return 32 * w + __ffs(mw) - 1;
            }
            return -1;
        };
        float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
        int cur = next_kept(-1);
        if (cur >= 0 && t < GT_BK) {
            const int64_t kb = hb + block_of(cb + cur) * GT_BK;
            if (kb + t < he) pre = __ldg(hits + kb + t);
        }
        while (cur >= 0 && !failed) {
            {
                const int64_t kb = hb + block_of(cb + cur) * GT_BK;
                done_hits += (he - kb) < GT_BK ? (he - kb) : GT_BK;
                // the block's hits (the previous block's panels are no longer read: its
                // MMAs completed before the barrier that ended its iteration)
                float4 *sh = reinterpret_cast<float4 *>(gsm + OFF_HITS);
                if (t < GT_BK) sh[t] = pre;
                __syncthreads();
                // panels
#pragma unroll 2
                for (int j = 0; j < GT_BK / 4; ++j) {
                    const int kc = 4 * j + lk;
                    const int64_t k = kb + kc;
                    float va0 = 0.f, va1 = 0.f, vb[NB];
#pragma unroll
                    for (int c = 0; c < NB; ++c) vb[c] = 0.f;
                    if (k < he) {
                        const float4 h = sh[kc];
                        // x - t_x z, y - t_y z with one rounding each, as grid_sep_kernel
                        const float u0 = __fmaf_rn(-t0a, h.z, h.x), u1 = __fmaf_rn(-t0b, h.z, h.x);
                        va0 = ex2_mufu(-(u0 * u0) * kk);
                        va1 = ex2_mufu(-(u1 * u1) * kk);
#pragma unroll
                        for (int c = 0; c < NB; ++c) {
                            const float v = __fmaf_rn(-t1[c], h.z, h.y);
                            vb[c] = ex2_mufu(-(v * v) * kk);
                        }
                    }
                    float hi, lo;
                    const int o0 = panel_off(m0, kc), o1 = panel_off(m1, kc);
                    split_tf32(va0, hi, lo);
                    *reinterpret_cast<float *>(gsm + OFF_AHI + o0) = hi;
                    *reinterpret_cast<float *>(gsm + OFF_ALO + o0) = lo;
                    split_tf32(va1, hi, lo);
                    *reinterpret_cast<float *>(gsm + OFF_AHI + o1) = hi;
                    *reinterpret_cast<float *>(gsm + OFF_ALO + o1) = lo;
#pragma unroll
                    for (int c = 0; c < NB; ++c) {
                        const int ob = panel_off(mb[c], kc);
                        split_tf32(vb[c], hi, lo);
                        *reinterpret_cast<float *>(gsm + OFF_BHI + ob) = hi;
                        *reinterpret_cast<float *>(gsm + OFF_BLO + ob) = lo;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (t == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = smem_addr(gsm);
#pragma unroll
                    for (int ks = 0; ks < GT_BK / 8; ++ks) {  // K = 8 per MMA: two core matrices
                        const uint64_t ah = gt_desc(base + OFF_AHI + ks * 256, 128, 1024);
                        const uint64_t al = gt_desc(base + OFF_ALO + ks * 256, 128, 1024);
                        const uint64_t bh = gt_desc(base + OFF_BHI + ks * 256, 128, 1024);
                        const uint64_t bl = gt_desc(base + OFF_BLO + ks * 256, 128, 1024);
                        gt_mma(tmem, ah, bh, L::IDESC, (any || ks > 0) ? 1u : 0u);
                        gt_mma(tmem, ah, bl, L::IDESC, 1u);
                        gt_mma(tmem, al, bh, L::IDESC, 1u);
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_addr)
                        : "memory");
                }
                any = true;
                const int nxt = next_kept(cur);
                pre = make_float4(0.f, 0.f, 0.f, 0.f);
                if (nxt >= 0 && t < GT_BK) {
                    const int64_t kn = hb + block_of(cb + nxt) * GT_BK;
                    if (kn + t < he) pre = __ldg(hits + kn + t);
                }
                // one thread waits for the MMAs (the others at the barrier, not polling shared memory)
                bool ok = true;
                if (t == 0) {
                    ok = gt_wait(bar_addr, phase);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                }
                phase ^= 1u;
                const bool all_ok = __syncthreads_and(ok);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (!all_ok) {
                    failed = true;
                    break;
                }
                cur = nxt;
            }
        }
    }
    if (failed) {
        if (t == 0) atomicExch(err, 1);
        gt_wait(bar_addr, phase ^ 1u);  // bounded: let the last MMAs finish before freeing TMEM
    } else {
        if (work && t == 0 && done_hits > 0) {
            const int64_t cw = (g.n0 - ti0 < GT_BM ? g.n0 - ti0 : GT_BM), ch = (g.n1 - tj0 < GT_BN ? g.n1 - tj0 : GT_BN);
            atomicAdd(work + RETINA_WORK_GRID, (unsigned long long)(done_hits * cw * ch));
        }
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (theta_0 cells) and
        // columns 128 (w / 4) .. + 127 (theta_1 cells)
        const int q = warp & 3, half = warp >> 2;
        const int i = ti0 + 32 * q + lane;
        float *dst = out + (int64_t)s * split_stride + (int64_t)e * event_stride;
#pragma unroll 1
        for (int part = 0; part < GT_BN / 64; ++part) {
            float v[32];
            if (any) {
                gt_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(GT_BN / 2 * half + 32 * part), v);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = 0.f;
            }
            if (i < g.n0) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int j = tj0 + GT_BN / 2 * half + 32 * part + c;
                    if (j < g.n1) dst[(int64_t)j * g.n0 + i] = v[c];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_NCOLS));
    }
}

template <int BN>
static cudaError_t launch_grid_tc_t(dim3 grid, cudaStream_t st, const float4 *hits, int64_t n_hits, const int64_t *off,
                                   const float4 *boxes, GridDev g, float kk, int splits, int tiles0, float *out,
                                   int64_t split_stride, int64_t event_stride, int32_t *err) {
    const size_t smem = GtLayout<BN>::SMEM;
    cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(grid_tc_kernel<BN>), smem);
    if (aerr != cudaSuccess) return aerr;
    PrioLaunch L(grid, dim3(GT_THREADS), smem, st, true);
    return cudaLaunchKernelEx(&L.cfg, grid_tc_kernel<BN>, hits, n_hits, off, boxes, g, kk, splits, tiles0, out,
                              split_stride, event_stride, work_counters(), err);
}

cudaError_t launch_grid_tc(int bn, dim3 grid, cudaStream_t st, const float4 *hits, int64_t n_hits, const int64_t *off,
                           const float4 *boxes, GridDev g, float kk, int splits, int tiles0, float *out,
                           int64_t split_stride, int64_t event_stride, int32_t *err) {
    return bn == 256 ? launch_grid_tc_t<256>(grid, st, hits, n_hits, off, boxes, g, kk, splits, tiles0, out,
                                             split_stride, event_stride, err)
                     : launch_grid_tc_t<128>(grid, st, hits, n_hits, off, boxes, g, kk, splits, tiles0, out,
                                             split_stride, event_stride, err);
}

}  // namespace retina
