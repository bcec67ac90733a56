// Learned seed proposer: slope histogram -> small conv net -> top-K seeds,
// with its training step (BCE with logits, backward, Adam).
//
// Network (per event, 64 x 64 pixels): conv 3x3 1 -> 16 + ReLU, conv 3x3
// 16 -> 32 + ReLU, 1x1 32 -> 1 (logits); 'same' zero padding, stride 1,
// cross-correlation.  Weights and activations are bfloat16 (round to nearest
// even); every sum accumulates in FP32.  Parameters are one FP32 master
// vector: W1 [16,1,3,3] at 0, b1 at 144, W2 [32,16,3,3] at 160, b2 at 4768,
// W3 [32] at 4800, b3 at 4832 (4833 values); the kernels read them rounded
// to bfloat16.
//
// Training: loss = mean over the batch's pixels of
//   pw y softplus(-z) + (1 - y) softplus(z),  pw = min(100, #neg / max(#pos, 1)),
// dL/dz = (pw y (sigmoid(z) - 1) + (1 - y) sigmoid(z)) / N; the gradient
// images dL/da2 and dL/da1 are stored as bfloat16.  Every reduction runs in a
// fixed order (per-CTA partials, then a fixed-order sum), so a training step
// is deterministic.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace retina {

constexpr int SN = 64, SN_PX = 4096, SC1 = 16, SC2 = 32;
constexpr int O_W1 = 0, O_B1 = 144, O_W2 = 160, O_B2 = 4768, O_W3 = 4800, O_B3 = 4832, NPAR = 4833;
constexpr int ROWS = 4;                  // image rows per CTA
constexpr int TILES = SN / ROWS;         // CTAs per event
constexpr int PART = NPAR + 1;           // per-CTA partial: gradient + loss sum
constexpr int SN_THREADS = 256;          // = ROWS * 64 pixels, one per thread

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// ---------------------------------------------------------------------------
// S7: slope histogram
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
slope_hist_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, float lo,
                  float scale, float zmin, uint16_t *__restrict__ feat, int32_t *__restrict__ counts_out) {
    __shared__ int cnt[SN_PX];
    const int e = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < SN_PX; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    for (int64_t k = hb + tid; k < he; k += blockDim.x) {
        const float4 h = __ldg(hits + k);
        if (!(fabsf(h.z) >= zmin)) continue;
        // decided in float32 exactly as written: u = x / z, bin = floor((u - lo) * scale)
        const float bu = floorf(__fmul_rn(__fsub_rn(__fdiv_rn(h.x, h.z), lo), scale));
        const float bv = floorf(__fmul_rn(__fsub_rn(__fdiv_rn(h.y, h.z), lo), scale));
        if (bu >= 0.f && bu < (float)SN && bv >= 0.f && bv < (float)SN) atomicAdd(&cnt[(int)bv * SN + (int)bu], 1);
    }
    __syncthreads();
    for (int i = tid; i < SN_PX; i += blockDim.x) {
        feat[(int64_t)e * SN_PX + i] = bf16_bits(log1pf((float)cnt[i]));
        if (counts_out) counts_out[(int64_t)e * SN_PX + i] = cnt[i];
    }
}

// ---------------------------------------------------------------------------
// S8: forward
// ---------------------------------------------------------------------------
// conv1 (1 -> 16) + ReLU for ROWS rows of one event; h1 stored bfloat16.
__global__ void __launch_bounds__(SN_THREADS)
conv1_kernel(const uint16_t *__restrict__ feat, const float *__restrict__ params, uint16_t *__restrict__ h1) {
    __shared__ float tile[ROWS + 2][SN + 2];
    __shared__ float w[O_W2];  // W1 (144) and b1 (16), bf16-rounded
    const int e = blockIdx.x, r0 = blockIdx.y * ROWS, tid = threadIdx.x;
    for (int i = tid; i < O_W2; i += SN_THREADS) w[i] = bf16r(params[i]);
    for (int i = tid; i < (ROWS + 2) * (SN + 2); i += SN_THREADS) {
        const int tr = i / (SN + 2), tc = i % (SN + 2);
        const int r = r0 - 1 + tr, c = tc - 1;
        tile[tr][tc] = (r >= 0 && r < SN && c >= 0 && c < SN) ? bf16_val(feat[(int64_t)e * SN_PX + r * SN + c]) : 0.f;
    }
    __syncthreads();
    const int rr = tid / SN, c = tid % SN;
    float x[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) x[t] = tile[rr + t / 3][c + t % 3];
#pragma unroll
    for (int o = 0; o < SC1; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc = __fmaf_rn(w[O_W1 + o * 9 + t], x[t], acc);
        acc += w[O_B1 + o];
        h1[((int64_t)e * SC1 + o) * SN_PX + (r0 + rr) * SN + c] = bf16_bits(fmaxf(acc, 0.f));
    }
}

// conv2 (16 -> 32) + ReLU + 1x1 head for ROWS rows of one event.
constexpr int CONV2_SMEM_FLOATS = SC1 * 9 * SC2 + SC2 + SC2 + 4 + SC1 * (ROWS + 2) * (SN + 2);

template <bool STORE_H2>
__global__ void __launch_bounds__(SN_THREADS)
conv2_head_kernel(const uint16_t *__restrict__ h1, const float *__restrict__ params, uint16_t *__restrict__ h2,
                  float *__restrict__ logits) {
    extern __shared__ __align__(16) float sm[];
    float *wT = sm;                                   // [i][t][o]: W2[o][i][t]
    float *b2 = wT + SC1 * 9 * SC2;
    float *w3 = b2 + SC2;
    float *b3 = w3 + SC2;
    float *tile = b3 + 4;                             // [i][ROWS + 2][SN + 2]
    const int e = blockIdx.x, r0 = blockIdx.y * ROWS, tid = threadIdx.x;
    for (int j = tid; j < SC1 * 9 * SC2; j += SN_THREADS) {
        const int o = j % SC2, it = j / SC2;         // it = i * 9 + t
        wT[j] = bf16r(params[O_W2 + o * SC1 * 9 + it]);
    }
    for (int j = tid; j < SC2; j += SN_THREADS) {
        b2[j] = bf16r(params[O_B2 + j]);
        w3[j] = bf16r(params[O_W3 + j]);
    }
    if (tid == 0) b3[0] = bf16r(params[O_B3]);
    for (int j = tid; j < SC1 * (ROWS + 2) * (SN + 2); j += SN_THREADS) {
        const int i = j / ((ROWS + 2) * (SN + 2)), rem = j % ((ROWS + 2) * (SN + 2));
        const int tr = rem / (SN + 2), tc = rem % (SN + 2);
        const int r = r0 - 1 + tr, c = tc - 1;
        tile[j] = (r >= 0 && r < SN && c >= 0 && c < SN) ? bf16_val(h1[((int64_t)e * SC1 + i) * SN_PX + r * SN + c])
                                                          : 0.f;
    }
    __syncthreads();
    const int rr = tid / SN, c = tid % SN;
    float acc[SC2];
#pragma unroll
    for (int o = 0; o < SC2; ++o) acc[o] = 0.f;
    for (int i = 0; i < SC1; ++i) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float xv = tile[(i * (ROWS + 2) + rr + t / 3) * (SN + 2) + c + t % 3];
            const float4 *wp = reinterpret_cast<const float4 *>(wT + (i * 9 + t) * SC2);
#pragma unroll
            for (int q = 0; q < SC2 / 4; ++q) {
                const float4 wv = wp[q];
                acc[4 * q + 0] = __fmaf_rn(wv.x, xv, acc[4 * q + 0]);
                acc[4 * q + 1] = __fmaf_rn(wv.y, xv, acc[4 * q + 1]);
                acc[4 * q + 2] = __fmaf_rn(wv.z, xv, acc[4 * q + 2]);
                acc[4 * q + 3] = __fmaf_rn(wv.w, xv, acc[4 * q + 3]);
            }
        }
    }
    float z = 0.f;
    const int64_t px = (int64_t)(r0 + rr) * SN + c;
#pragma unroll
    for (int o = 0; o < SC2; ++o) {
        const float hv = bf16r(fmaxf(acc[o] + b2[o], 0.f));
        if (STORE_H2) h2[((int64_t)e * SC2 + o) * SN_PX + px] = bf16_bits(hv);
        z = __fmaf_rn(w3[o], hv, z);
    }
    logits[(int64_t)e * SN_PX + px] = z + b3[0];
}

// ---------------------------------------------------------------------------
// S10: training step
// ---------------------------------------------------------------------------
__global__ void count_pos_kernel(const uint8_t *__restrict__ labels, int64_t n, unsigned long long *__restrict__ npos) {
    __shared__ unsigned long long part[8];
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += labels[i] ? 1ull : 0ull;
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(npos, s);  // integer sum: order-independent
    }
}

constexpr int BWD_D2 = SC2 * (ROWS + 2) * (SN + 2);      // dL/da2 tile with halo
constexpr int BWD_H1 = SC1 * (ROWS + 2) * (SN + 2);      // h1 tile with halo
constexpr int BWD_X = (ROWS + 2) * (SN + 2);             // input tile with halo
constexpr int BWD_D1 = SC1 * ROWS * SN;                  // dL/da1, own rows
constexpr int BWD_W2 = SC2 * SC1 * 9;
constexpr int BWD_SCR = SN_THREADS * SC2;                // per-pixel scratch for ordered sums
constexpr int BWD_SMEM_FLOATS = BWD_W2 + SC2 + BWD_D2 + BWD_H1 + BWD_X + BWD_D1 + BWD_SCR + SN_THREADS;

__device__ __forceinline__ float softplusf(float t) { return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t)); }

// One CTA per (event, ROWS rows): loss, head, conv2 and conv1 gradients of
// its own pixels, written as one partial vector (sums in a fixed order).
__global__ void __launch_bounds__(SN_THREADS)
seednet_backward_kernel(const uint16_t *__restrict__ feat, const uint16_t *__restrict__ h1,
                        const uint16_t *__restrict__ h2, const float *__restrict__ logits,
                        const uint8_t *__restrict__ labels, const float *__restrict__ params,
                        const unsigned long long *__restrict__ npos_ptr, int64_t n_px_total,
                        float *__restrict__ partials) {
    extern __shared__ __align__(16) float sm[];
    float *w2 = sm;                      // [o][i][t]
    float *w3 = w2 + BWD_W2;
    float *d2 = w3 + SC2;                // [o][ROWS+2][SN+2]
    float *ht = d2 + BWD_D2;             // [i][ROWS+2][SN+2]
    float *xt = ht + BWD_H1;             // [ROWS+2][SN+2]
    float *d1 = xt + BWD_X;              // [i][ROWS][SN]
    float *scr = d1 + BWD_D1;            // [SC2][SN_THREADS] per-pixel terms
    float *scr1 = scr + BWD_SCR;         // [SN_THREADS]
    const int e = blockIdx.x, r0 = blockIdx.y * ROWS, tid = threadIdx.x;
    float *out = partials + ((int64_t)e * TILES + blockIdx.y) * PART;
    const float npos = (float)*npos_ptr;
    const float pw = fminf(100.f, ((float)n_px_total - npos) / fmaxf(npos, 1.f));
    const float inv_n = 1.f / (float)n_px_total;

    for (int j = tid; j < BWD_W2; j += SN_THREADS) w2[j] = bf16r(params[O_W2 + j]);
    for (int j = tid; j < SC2; j += SN_THREADS) w3[j] = bf16r(params[O_W3 + j]);
    __syncthreads();
    // dL/da2 on the tile and its halo rows (zero outside the image)
    for (int j = tid; j < (ROWS + 2) * (SN + 2); j += SN_THREADS) {
        const int tr = j / (SN + 2), tc = j % (SN + 2);
        const int r = r0 - 1 + tr, c = tc - 1;
        const bool in = r >= 0 && r < SN && c >= 0 && c < SN;
        float dz = 0.f;
        const int64_t px = (int64_t)r * SN + c;
        if (in) {
            const float z = logits[(int64_t)e * SN_PX + px];
            const float y = labels[(int64_t)e * SN_PX + px] ? 1.f : 0.f;
            const float sg = 1.f / (1.f + expf(-z));
            dz = (pw * y * (sg - 1.f) + (1.f - y) * sg) * inv_n;
        }
        for (int o = 0; o < SC2; ++o) {
            float v = 0.f;
            if (in && bf16_val(h2[((int64_t)e * SC2 + o) * SN_PX + px]) > 0.f) v = bf16r(dz * w3[o]);
            d2[(o * (ROWS + 2) + tr) * (SN + 2) + tc] = v;
        }
    }
    for (int j = tid; j < BWD_H1; j += SN_THREADS) {
        const int i = j / ((ROWS + 2) * (SN + 2)), rem = j % ((ROWS + 2) * (SN + 2));
        const int tr = rem / (SN + 2), tc = rem % (SN + 2);
        const int r = r0 - 1 + tr, c = tc - 1;
        ht[j] = (r >= 0 && r < SN && c >= 0 && c < SN) ? bf16_val(h1[((int64_t)e * SC1 + i) * SN_PX + r * SN + c]) : 0.f;
    }
    for (int j = tid; j < BWD_X; j += SN_THREADS) {
        const int tr = j / (SN + 2), tc = j % (SN + 2);
        const int r = r0 - 1 + tr, c = tc - 1;
        xt[j] = (r >= 0 && r < SN && c >= 0 && c < SN) ? bf16_val(feat[(int64_t)e * SN_PX + r * SN + c]) : 0.f;
    }
    __syncthreads();

    // ---- own pixel: loss term, head terms, dL/dh1 -> dL/da1
    const int rr = tid / SN, c = tid % SN;
    const int64_t px = (int64_t)(r0 + rr) * SN + c;
    {
        const float z = logits[(int64_t)e * SN_PX + px];
        const float y = labels[(int64_t)e * SN_PX + px] ? 1.f : 0.f;
        const float sg = 1.f / (1.f + expf(-z));
        const float dz = (pw * y * (sg - 1.f) + (1.f - y) * sg) * inv_n;
        scr1[tid] = pw * y * softplusf(-z) + (1.f - y) * softplusf(z);
        for (int o = 0; o < SC2; ++o) scr[o * SN_THREADS + tid] = dz * bf16_val(h2[((int64_t)e * SC2 + o) * SN_PX + px]);
        // head bias gradient uses dz: kept in d1's last use below via a separate pass
        float dh[SC1];
#pragma unroll
        for (int i = 0; i < SC1; ++i) dh[i] = 0.f;
        for (int o = 0; o < SC2; ++o) {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                // a2[o][r'][c'] uses h1[i][r' + dy - 1][c' + dx - 1]: r' = r - dy + 1
                const int dy = t / 3, dx = t % 3;
                const float dv = d2[(o * (ROWS + 2) + rr + 2 - dy) * (SN + 2) + c + 2 - dx];
#pragma unroll
                for (int i = 0; i < SC1; ++i) dh[i] = __fmaf_rn(w2[(o * SC1 + i) * 9 + t], dv, dh[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < SC1; ++i) {
            const bool on = ht[(i * (ROWS + 2) + rr + 1) * (SN + 2) + c + 1] > 0.f;
            d1[(i * ROWS + rr) * SN + c] = on ? bf16r(dh[i]) : 0.f;
        }
    }
    __syncthreads();

    // ---- ordered sums, one output per thread (loops over own pixels in order)
    // loss and head
    if (tid == 0) {
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) s += scr1[p];
        out[NPAR] = s;
    }
    if (tid < SC2) {
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) s += scr[tid * SN_THREADS + p];
        out[O_W3 + tid] = s;
    }
    if (tid == 64) {  // b3: sum of dz = sum over pixels recomputed in order
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) {
            const int64_t q = (int64_t)(r0 + p / SN) * SN + p % SN;
            const float z = logits[(int64_t)e * SN_PX + q];
            const float y = labels[(int64_t)e * SN_PX + q] ? 1.f : 0.f;
            const float sg = 1.f / (1.f + expf(-z));
            s += (pw * y * (sg - 1.f) + (1.f - y) * sg) * inv_n;
        }
        out[O_B3] = s;
    }
    // conv2 weights: dW2[o][i][t] = sum_px d2[o][px] h1[i][px + t - 1]; b2[o] = sum_px d2[o][px]
    for (int j = tid; j < BWD_W2; j += SN_THREADS) {
        const int o = j / (SC1 * 9), i = (j / 9) % SC1, t = j % 9, dy = t / 3, dx = t % 3;
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) {
            const int pr = p / SN, pc = p % SN;
            s = __fmaf_rn(d2[(o * (ROWS + 2) + pr + 1) * (SN + 2) + pc + 1],
                          ht[(i * (ROWS + 2) + pr + dy) * (SN + 2) + pc + dx], s);
        }
        out[O_W2 + j] = s;
    }
    if (tid < SC2) {
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) s += d2[(tid * (ROWS + 2) + p / SN + 1) * (SN + 2) + p % SN + 1];
        out[O_B2 + tid] = s;
    }
    // conv1 weights: dW1[o][t] = sum_px d1[o][px] x[px + t - 1]; b1[o] = sum_px d1[o][px]
    for (int j = tid; j < SC1 * 9; j += SN_THREADS) {
        const int o = j / 9, t = j % 9, dy = t / 3, dx = t % 3;
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) {
            const int pr = p / SN, pc = p % SN;
            s = __fmaf_rn(d1[(o * ROWS + pr) * SN + pc], xt[(pr + dy) * (SN + 2) + pc + dx], s);
        }
        out[O_W1 + j] = s;
    }
    if (tid >= 96 && tid < 96 + SC1) {
        const int o = tid - 96;
        float s = 0.f;
        for (int p = 0; p < SN_THREADS; ++p) s += d1[(o * ROWS + p / SN) * SN + p % SN];
        out[O_B1 + o] = s;
    }
}

// grad[j] = sum over CTAs of partials[cta][j], in CTA order; loss likewise / N.
__global__ void reduce_partials_seednet(const float *__restrict__ partials, int n_cta, int64_t n_px_total,
                                        float *__restrict__ grad, float *__restrict__ loss) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > NPAR) return;
    float s = 0.f;
    for (int k = 0; k < n_cta; ++k) s += partials[(int64_t)k * PART + j];
    if (j < NPAR)
        grad[j] = s;
    else if (loss)
        *loss = s / (float)n_px_total;
}

__global__ void adam_kernel(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NPAR) return;
    const float g = grad[j];
    const float mj = b1 * m[j] + (1.f - b1) * g;
    const float vj = b2 * v[j] + (1.f - b2) * g * g;
    m[j] = mj;
    v[j] = vj;
    params[j] -= lr * (mj * c1) / (sqrtf(vj * c2) + eps);
}

// ---------------------------------------------------------------------------
// S9: top-K seeds
// ---------------------------------------------------------------------------
// One CTA (1024 threads) per event.  Cells are ranked by logit (bitonic sort
// of (order key, index)); with hits, the first R_MAX ranked cells are split
// into SUB x SUB sub-cells: pass 1 counts each sub-cell's hits, a block scan
// hands out seed slots (one per sub-cell with >= n_min hits, fullest first;
// else one for the fullest non-empty sub-cell; else the cell centre), pass 2
// sums the in-sub-cell positions of the hits of every slot (2^-32 fixed
// point, integer atomics: order-independent), and each slot's seed is its
// hits' mean slope.
constexpr int SUB = 4, R_MAX = 1024, PROP_THREADS = 1024;
static_assert(R_MAX == PROP_THREADS, "one thread per splittable ranked cell");
constexpr float FRAC_ONE = 4294967296.f;  // 2^32

size_t propose_smem_bytes(int K) {
    return (size_t)SN_PX * 8 + (size_t)K * 16 + (size_t)R_MAX * SUB * SUB * 4 + (size_t)K * 12 + 64 * 4 +
           (size_t)SN_PX * 2;
}

// sub-cell (fine) bins of a hit, float32 as the histogram: t = (u - lo) * (4 s)
__device__ __forceinline__ bool fine_bins(const float4 h, float lo, float s4, float zmin, float &tu, float &tv,
                                          int &fu, int &fv) {
    if (!(fabsf(h.z) >= zmin)) return false;
    tu = __fmul_rn(__fsub_rn(__fdiv_rn(h.x, h.z), lo), s4);
    tv = __fmul_rn(__fsub_rn(__fdiv_rn(h.y, h.z), lo), s4);
    const float bu = floorf(tu), bv = floorf(tv);
    if (!(bu >= 0.f && bu < (float)(SN * SUB) && bv >= 0.f && bv < (float)(SN * SUB))) return false;
    fu = (int)bu;
    fv = (int)bv;
    return true;
}

__global__ void __launch_bounds__(PROP_THREADS)
propose_seeds_kernel(const float *__restrict__ logits, int K, float lo, float w, float scale, float zmin, int n_min,
                     const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                     float *__restrict__ seeds, int32_t *__restrict__ idx_out) {
    extern __shared__ __align__(16) unsigned char psm[];
    uint64_t *keys = reinterpret_cast<uint64_t *>(psm);                          // [4096]
    unsigned long long *s_sum = reinterpret_cast<unsigned long long *>(keys + SN_PX);  // [K][2]
    int *sub = reinterpret_cast<int *>(s_sum + 2 * (size_t)K);                   // [R_MAX][16]: counts, then slots
    int *s_cnt = sub + R_MAX * SUB * SUB;                                        // [K]
    int *s_cell = s_cnt + K;                                                     // [K]
    int *s_fine = s_cell + K;                                                    // [K]: fine bin, -1 = centre
    int *scan = s_fine + K;                                                      // [64]
    int16_t *rank = reinterpret_cast<int16_t *>(scan + 64);                      // [4096]
    const int e = blockIdx.x, tid = threadIdx.x;
    const float s4 = scale * (float)SUB;
    // rank the cells: thread t holds cells 4t .. 4t+3, sorted in registers
    // (bitonic; shuffles and shared memory for the wider strides)
    constexpr int KPT = SN_PX / PROP_THREADS;
    static_assert(KPT == 4, "four cells per thread");
    uint64_t kv[KPT];
    {
        const float4 z4 = reinterpret_cast<const float4 *>(logits + (int64_t)e * SN_PX)[tid];
        const float zz[KPT] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int r = 0; r < KPT; ++r) {
            const int i = tid * KPT + r;
            const float z = zz[r] + 0.f;                                 // -0 -> +0: equal logits tie
            const uint32_t k = isnan(z) ? 0u : float_order_key(z);      // NaN ranks below every number
            kv[r] = ((uint64_t)(~k) << 32) | (uint32_t)i;                // larger z first, then lower index
        }
    }
    for (int i = tid; i < R_MAX * SUB * SUB; i += PROP_THREADS) sub[i] = 0;
    bitonic_sort_regs<uint64_t, KPT, PROP_THREADS>(kv, keys);
    __syncthreads();  // the sort's last shared-memory reads are done before keys is overwritten
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        keys[tid * KPT + r] = kv[r];
        rank[(int)(uint32_t)kv[r]] = (int16_t)(tid * KPT + r);
    }
    __syncthreads();
    int64_t hb = 0, he = 0;
    if (hits) event_range(off, n_hits, e, hb, he);
    // pass 1: hits per sub-cell of the first R_MAX ranked cells
    for (int64_t k = hb + tid; k < he; k += PROP_THREADS) {
        float tu, tv;
        int fu, fv;
        if (!fine_bins(__ldg(hits + k), lo, s4, zmin, tu, tv, fu, fv)) continue;
        const int r = rank[(fv / SUB) * SN + fu / SUB];
        if (r < R_MAX) atomicAdd(&sub[r * SUB * SUB + (fv % SUB) * SUB + fu % SUB], 1);
    }
    __syncthreads();
    // schedule: thread r owns ranked cell r (< R_MAX = blockDim)
    const int r = tid;
    const int cell_r = (int)(uint32_t)keys[r];
    int cnt[SUB * SUB];
    int nq = 0, best = -1, best_cnt = 0;
#pragma unroll
    for (int q = 0; q < SUB * SUB; ++q) {
        cnt[q] = sub[r * SUB * SUB + q];
        nq += cnt[q] >= n_min;
        if (cnt[q] > best_cnt) {  // strict: the lowest sub-cell index wins ties
            best = q;
            best_cnt = cnt[q];
        }
    }
    const int thr = nq > 0 ? n_min : (best >= 0 ? best_cnt : INT32_MAX);
    const int e_r = nq > 0 ? nq : 1;
    // block exclusive scan of e_r
    int incl = e_r;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) scan[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = scan[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        scan[32 + lane] = t;  // inclusive scan of the warp totals
    }
    __syncthreads();
    const int off_r = (wid > 0 ? scan[32 + wid - 1] : 0) + incl - e_r;
    const int total_split = scan[32 + 31];
    // slots: sub-cells of ranked cell r in order (most hits, then lower index)
    int k_out = 0;
#pragma unroll
    for (int q = 0; q < SUB * SUB; ++q) {
        int slot = -1;
        if (cnt[q] >= thr && (nq > 0 || q == best)) {
            int pos = 0;
#pragma unroll
            for (int q2 = 0; q2 < SUB * SUB; ++q2)
                pos += (cnt[q2] >= thr && (nq > 0 || q2 == best)) &&
                       (cnt[q2] > cnt[q] || (cnt[q2] == cnt[q] && q2 < q));
            const int sl = off_r + pos;
            if (sl < K) {
                slot = sl;
                s_cell[sl] = cell_r;
                s_fine[sl] = ((cell_r / SN) * SUB + q / SUB) * (SN * SUB) + (cell_r % SN) * SUB + q % SUB;
                s_cnt[sl] = 0;
                s_sum[2 * sl] = s_sum[2 * sl + 1] = 0ull;
            }
            ++k_out;
        }
        sub[r * SUB * SUB + q] = slot;  // every thread read its own counts above
    }
    if (k_out == 0 && off_r < K) {  // empty cell: its centre
        s_cell[off_r] = cell_r;
        s_fine[off_r] = -1;
    }
    // cells ranked past R_MAX: their centres
    for (int q = R_MAX + tid; q < SN_PX; q += PROP_THREADS) {
        const int sl = total_split + (q - R_MAX);
        if (sl < K) {
            s_cell[sl] = (int)(uint32_t)keys[q];
            s_fine[sl] = -1;
        }
    }
    __syncthreads();
    // pass 2: position sums of each slot's hits
    for (int64_t k = hb + tid; k < he; k += PROP_THREADS) {
        float tu, tv;
        int fu, fv;
        if (!fine_bins(__ldg(hits + k), lo, s4, zmin, tu, tv, fu, fv)) continue;
        const int rr = rank[(fv / SUB) * SN + fu / SUB];
        if (rr >= R_MAX) continue;
        const int sl = sub[rr * SUB * SUB + (fv % SUB) * SUB + fu % SUB];
        if (sl < 0) continue;
        atomicAdd(&s_cnt[sl], 1);  // t - floor(t) is exact in float32; scaling by 2^32 is exact
        atomicAdd(&s_sum[2 * sl], (unsigned long long)__float2ll_rn(__fsub_rn(tu, (float)fu) * FRAC_ONE));
        atomicAdd(&s_sum[2 * sl + 1], (unsigned long long)__float2ll_rn(__fsub_rn(tv, (float)fv) * FRAC_ONE));
    }
    __syncthreads();
    for (int q = tid; q < K; q += PROP_THREADS) {
        const int64_t o = (int64_t)e * K + q;
        const int c = s_cell[q], f = s_fine[q], n = s_cnt[q];
        float su, sv;
        if (f >= 0 && n > 0) {  // mean slope: lo + (fine bin + mean frac) / (4 s), in double, rounded once
            const double dn = (double)n;
            su = (float)((double)lo + ((double)(f % (SN * SUB)) + (double)s_sum[2 * q] / dn * 0x1p-32) / (double)s4);
            sv = (float)((double)lo + ((double)(f / (SN * SUB)) + (double)s_sum[2 * q + 1] / dn * 0x1p-32) /
                                          (double)s4);
        } else {
            su = __fmaf_rn((float)(c % SN) + 0.5f, w, lo);
            sv = __fmaf_rn((float)(c / SN) + 0.5f, w, lo);
        }
        seeds[2 * o] = su;
        seeds[2 * o + 1] = sv;
        if (idx_out) idx_out[o] = c;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static float hist_scale(float lo, float hi) { return (float)((double)SN / ((double)hi - (double)lo)); }

cudaError_t launch_slope_hist(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, float lo, float hi,
                              float zmin, uint16_t *feat, int32_t *counts, cudaStream_t st) {
    slope_hist_kernel<<<n_events, 256, 0, st>>>(hits, n_hits, off, lo, hist_scale(lo, hi), zmin, feat, counts);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seednet_forward(const uint16_t *feat, int n_events, const float *params, float *logits,
                                   uint16_t *h1, uint16_t *h2, cudaStream_t st) {
    dim3 grid(n_events, TILES);
    conv1_kernel<<<grid, SN_THREADS, 0, st>>>(feat, params, h1);
    count_launches(1);
    cudaError_t err;
    if (option_value(RETINA_OPT_SEEDNET_TC)) {
        int32_t *flag = device_error_flag();
        if (!flag) return cudaErrorInvalidSymbol;
        return launch_conv2_head_tc(h1, n_events, params, h2, logits, flag, st);
    }
    const size_t smem = (size_t)CONV2_SMEM_FLOATS * sizeof(float);
    if (h2) {
        err = ensure_dynamic_smem(reinterpret_cast<const void *>(conv2_head_kernel<true>), smem);
        if (err != cudaSuccess) return err;
        conv2_head_kernel<true><<<grid, SN_THREADS, smem, st>>>(h1, params, h2, logits);
    } else {
        err = ensure_dynamic_smem(reinterpret_cast<const void *>(conv2_head_kernel<false>), smem);
        if (err != cudaSuccess) return err;
        conv2_head_kernel<false><<<grid, SN_THREADS, smem, st>>>(h1, params, nullptr, logits);
    }
    count_launches(1);
    return cudaGetLastError();
}

// workspace of a training step: h1, h2 (bf16), logits, per-CTA partials, grad, positives counter
struct TrainWs {
    size_t h1, h2, logits, partials, grad, npos, total;
};

static size_t r256(size_t v) { return (v + 255) / 256 * 256; }

static TrainWs train_ws(int n_events) {
    TrainWs w;
    size_t o = 0;
    w.h1 = o;
    o += r256((size_t)n_events * SC1 * SN_PX * 2);
    w.h2 = o;
    o += r256((size_t)n_events * SC2 * SN_PX * 2);
    w.logits = o;
    o += r256((size_t)n_events * SN_PX * 4);
    w.partials = o;
    o += r256((size_t)n_events * TILES * PART * 4);
    w.grad = o;
    o += r256((size_t)NPAR * 4);
    w.npos = o;
    o += 256;
    w.total = o;
    return w;
}

size_t seednet_train_ws_bytes(int n_events) { return train_ws(n_events).total; }

cudaError_t launch_seednet_train_step(const uint16_t *feat, const uint8_t *labels, int n_events, float *params,
                                      float *m, float *v, int step, float lr, float b1, float b2, float eps,
                                      float *loss_out, float *grad_out, void *ws, cudaStream_t st) {
    const TrainWs w = train_ws(n_events);
    char *base = (char *)ws;
    uint16_t *h1 = (uint16_t *)(base + w.h1);
    uint16_t *h2 = (uint16_t *)(base + w.h2);
    float *logits = (float *)(base + w.logits);
    float *partials = (float *)(base + w.partials);
    float *grad = grad_out ? grad_out : (float *)(base + w.grad);
    unsigned long long *npos = (unsigned long long *)(base + w.npos);
    const int64_t n_px = (int64_t)n_events * SN_PX;
    cudaError_t err = cudaMemsetAsync(npos, 0, sizeof(unsigned long long), st);
    if (err != cudaSuccess) return err;
    count_pos_kernel<<<sm_count() * 4, 256, 0, st>>>(labels, n_px, npos);
    err = launch_seednet_forward(feat, n_events, params, logits, h1, h2, st);
    if (err != cudaSuccess) return err;
    const size_t smem = (size_t)BWD_SMEM_FLOATS * sizeof(float);
    err = ensure_dynamic_smem(reinterpret_cast<const void *>(seednet_backward_kernel), smem);
    if (err != cudaSuccess) return err;
    seednet_backward_kernel<<<dim3(n_events, TILES), SN_THREADS, smem, st>>>(feat, h1, h2, logits, labels, params,
                                                                           npos, n_px, partials);
    reduce_partials_seednet<<<(NPAR + 1 + 255) / 256, 256, 0, st>>>(partials, n_events * TILES, n_px, grad,
                                                                     loss_out);
    count_launches(3);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_seednet_adam(params, m, v, grad, step, lr, b1, b2, eps, st);
}

cudaError_t launch_seednet_adam(float *params, float *m, float *v, const float *grad, int step, float lr, float b1,
                                float b2, float eps, cudaStream_t st) {
    // bias corrections 1 / (1 - beta^step), in double, rounded once
    const double c1 = 1.0 / (1.0 - pow((double)b1, (double)step));
    const double c2 = 1.0 / (1.0 - pow((double)b2, (double)step));
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(params, m, v, grad, lr, b1, b2, eps, (float)c1, (float)c2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_propose_seeds(const float *logits, int n_events, int K, float lo, float hi, float zmin, int n_min,
                                 const float4 *hits, int64_t n_hits, const int64_t *off, float *seeds, int32_t *idx,
                                 cudaStream_t st) {
    const float w = (float)(((double)hi - (double)lo) / SN);
    const size_t smem = propose_smem_bytes(K);
    cudaError_t err = ensure_dynamic_smem(reinterpret_cast<const void *>(propose_seeds_kernel), smem);
    if (err != cudaSuccess) return err;
    propose_seeds_kernel<<<n_events, PROP_THREADS, smem, st>>>(logits, K, lo, w, hist_scale(lo, hi), zmin, n_min,
                                                               hits, n_hits, off, seeds, idx);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
