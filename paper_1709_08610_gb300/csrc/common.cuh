// Device-side helpers shared by the retina kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "retina.h"

namespace retina {

// log2(e): exp(-a) = 2^(-a * log2(e)); the bandwidth factor folds it in on the host.
constexpr double kLog2e = 1.4426950408889634073599246810019;

struct GridDev {
    float lo0, lo1, step0, step1;
    int n0, n1;
};

// 2^x on the MUFU (SFU) pipe, denormal results flushed to zero.
__device__ __forceinline__ float ex2_mufu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 fused multiply-add, round-to-nearest per lane (each lane is
// bitwise the scalar __fmaf_rn): acc = a * b + acc on {lo, hi} pairs.
__device__ __forceinline__ void ffma2_rn(unsigned long long &acc, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

// Butterfly (xor) sum: every lane ends with the bitwise-identical total,
// because each level adds the same two operands in either order.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Order-preserving map of a float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t float_order_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Hit range [hb, he) of event e with both offsets clamped to [0, n_hits]; a
// decreasing pair gives an empty event.
__device__ __forceinline__ void event_range(const int64_t *__restrict__ off, int64_t n_hits, int e, int64_t &hb,
                                            int64_t &he) {
    int64_t a = off[e], b = off[e + 1];
    a = a < 0 ? 0 : (a > n_hits ? n_hits : a);
    b = b < a ? a : (b > n_hits ? n_hits : b);
    hb = a;
    he = b;
}

__device__ __forceinline__ float cell_centre(float lo, float step, int i) {
    // lo + (i + 1/2) step; exact for step = 2^-k and |i| < 2^23
    return __fmaf_rn((float)i + 0.5f, step, lo);
}

}  // namespace retina
