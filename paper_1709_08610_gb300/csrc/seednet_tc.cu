// Second convolution of the seed network (16 -> 32 channels, 3 x 3) plus the
// 1 x 1 head on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The layer is an implicit GEMM: for a tile of 128 pixels (two image rows),
//   a2[m][o] = sum over taps t = (dy, dx) of sum_k h1[k][pixel(m) + t - 1] W2[o][k][t]
// i.e. nine MMAs of M = 128 pixels, N = 32 output channels, K = 16 input
// channels, BF16 operands, FP32 accumulation in tensor memory (TMEM).
//   A_t (128 x 16, K-major): the tap-shifted pixels' 16 channels, copied per
//        tile from a zero-padded halo of h1 into the canonical no-swizzle
//        core-matrix layout (8 rows x 16 bytes per core matrix);
//   B_t (32 x 16, K-major): W2[:, :, t] rounded to bfloat16, once per CTA;
//   D   (128 x 32 FP32): TMEM lanes 0..127 = pixels, 32 columns = channels.
// One thread issues the MMAs and commits them to an mbarrier; every thread
// then reads its pixel's 32 sums (warp w reads TMEM lanes 32w..32w+31) and
// applies bias, ReLU, bfloat16 rounding and the head exactly as the CUDA-core
// kernel does.  Only the order in which the FP32 sums of a2 accumulate
// differs.  All waits are bounded: on a timeout the kernel records an error,
// waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace retina {

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_NCOLS = 32;                  // TMEM columns (the 32 output channels)
constexpr int A_BYTES = 128 * 16 * 2;         // one tap's A operand
constexpr int B_BYTES = 32 * 16 * 2;          // one tap's B operand
constexpr int HALO_BYTES = 4 * 66 * 16 * 2;   // rows r0-1..r0+2, cols -1..64, 16 channels
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + 9 * A_BYTES;
constexpr int OFF_HALO = OFF_B + 9 * B_BYTES;
constexpr int OFF_PAR = OFF_HALO + HALO_BYTES;        // b2[32], w3[32], b3
constexpr int OFF_BAR = OFF_PAR + 68 * 4;             // mbarrier (8 B) + TMEM address (4 B)
constexpr int TC_SMEM = OFF_BAR + 16;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle; lbo = byte distance between
// core matrices along K, sbo = along M / N; version 1 (bit 46)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
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

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(addr, parity)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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

__device__ __forceinline__ uint16_t bf16_bits_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

}  // namespace

// One CTA of 128 threads loops over tiles (event, pair of image rows).
template <bool STORE_H2>
__global__ void __launch_bounds__(TC_THREADS)
conv2_head_tc_kernel(const uint16_t *__restrict__ h1, const float *__restrict__ params, uint16_t *__restrict__ h2,
                     float *__restrict__ logits, int n_tiles, int32_t *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + OFF_A;
    unsigned char *sB = sm + OFF_B;
    uint16_t *halo = reinterpret_cast<uint16_t *>(sm + OFF_HALO);
    float *par = reinterpret_cast<float *>(sm + OFF_PAR);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_addr = smem_u32(bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_addr), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B_t[n][k] = bf16(W2[n][k][t]) in core-matrix layout: t*1024 + (n/8)*256 + (k/8)*128 + (n%8)*16 + (k%8)*2
    for (int idx = tid; idx < 9 * 32 * 16; idx += TC_THREADS) {
        const int t = idx / 512, n = (idx >> 4) & 31, k = idx & 15;
        const uint16_t v = bf16_bits_rn(params[160 + n * 144 + k * 9 + t]);
        *reinterpret_cast<uint16_t *>(sB + t * B_BYTES + (n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 +
                                      (k & 7) * 2) = v;
    }
    if (tid < 32) {
        par[tid] = bf16_round(params[4768 + tid]);       // b2
        par[32 + tid] = bf16_round(params[4800 + tid]);  // W3
    }
    if (tid == 0) par[64] = bf16_round(params[4832]);    // b3
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t phase = 0;
    bool failed = false;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int e = tile >> 5, r0 = (tile & 31) * 2;
        // halo[hr][hc][ch] (rows r0-1..r0+2, cols -1..64), zero outside the image: each item is
        // one pixel's 8-channel group, gathered from the 8 channel planes (loads coalesced along
        // the columns) and stored as one 16-byte vector
        for (int idx = tid; idx < 4 * 2 * 66; idx += TC_THREADS) {
            // lanes take consecutive 16-byte chunks (pixel, channel group): conflict-free stores
            const int grp = idx & 1, hc = (idx >> 1) % 66, hr = (idx >> 1) / 66;
            const int r = r0 - 1 + hr, c = hc - 1;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (r >= 0 && r < 64 && c >= 0 && c < 64) {
                const uint16_t *src = h1 + (((int64_t)e * 16 + 8 * grp) * 64 + r) * 64 + c;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = (uint32_t)src[(2 * q) * 4096] | ((uint32_t)src[(2 * q + 1) * 4096] << 16);
            }
            *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(halo) + (hr * 66 + hc) * 32 + grp * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
        __syncthreads();
        // A_t[m][8j..8j+7] = halo[(m/64 + dy)][(m%64 + dx)][8j..8j+7], 16-byte chunks
        for (int idx = tid; idx < 9 * 128 * 2; idx += TC_THREADS) {
            const int t = idx >> 8, m = (idx >> 1) & 127, j = idx & 1;
            const int dy = t / 3, dx = t - 3 * dy;
            const uint4 v = *reinterpret_cast<const uint4 *>(
                reinterpret_cast<const unsigned char *>(halo) + (((m >> 6) + dy) * 66 + (m & 63) + dx) * 32 + j * 16);
            *reinterpret_cast<uint4 *>(sA + t * A_BYTES + (m >> 3) * 256 + j * 128 + (m & 7) * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const uint64_t ad = smem_desc(smem_u32(sA + t * A_BYTES), 128, 256);
                const uint64_t bd = smem_desc(smem_u32(sB + t * B_BYTES), 128, 256);
                const uint32_t acc = t > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar_addr)
                         : "memory");
        }
        // one thread waits for the MMAs (the others at the barrier, not polling shared memory)
        bool ok = true;
        if (tid == 0) {
            ok = mbar_wait(bar_addr, phase);
            tc_fence_before();
        }
        phase ^= 1u;
        const bool all_ok = __syncthreads_and(ok);
        tc_fence_after();
        if (!all_ok) {  // every thread leaves together
            failed = true;
            break;
        }
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), acc);
        const int m = 32 * warp + lane;
        const int px = (r0 + (m >> 6)) * 64 + (m & 63);
        float z = 0.f;
#pragma unroll
        for (int o = 0; o < 32; ++o) {
            const float hv = bf16_round(fmaxf(acc[o] + par[o], 0.f));
            if (STORE_H2) h2[((int64_t)e * 32 + o) * 4096 + px] = bf16_bits_rn(hv);
            z = __fmaf_rn(par[32 + o], hv, z);
        }
        logits[(int64_t)e * 4096 + px] = z + par[64];
        tc_fence_before();
        __syncthreads();  // TMEM read and shared operands free before the next tile
    }
    if (failed) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait(bar_addr, phase ^ 1u);  // bounded: let the last MMAs finish before freeing TMEM
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NCOLS));
    }
}

cudaError_t launch_conv2_head_tc(const uint16_t *h1, int n_events, const float *params, uint16_t *h2, float *logits,
                                 int32_t *err, cudaStream_t st) {
    const int n_tiles = n_events * 32;
    int grid = sm_count() * 4;
    if (grid > n_tiles) grid = n_tiles;
    cudaError_t e;
    if (h2) {
        e = ensure_dynamic_smem(reinterpret_cast<const void *>(conv2_head_tc_kernel<true>), TC_SMEM);
        if (e != cudaSuccess) return e;
        conv2_head_tc_kernel<true><<<grid, TC_THREADS, TC_SMEM, st>>>(h1, params, h2, logits, n_tiles, err);
    } else {
        e = ensure_dynamic_smem(reinterpret_cast<const void *>(conv2_head_tc_kernel<false>), TC_SMEM);
        if (e != cudaSuccess) return e;
        conv2_head_tc_kernel<false><<<grid, TC_THREADS, TC_SMEM, st>>>(h1, params, nullptr, logits, n_tiles, err);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
