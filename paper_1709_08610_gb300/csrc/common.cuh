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

// Programmatic dependent launch: a kernel launched with the
// programmatic-serialization attribute may start while the previous kernel in
// its stream finishes; it must wait (pdl_wait) before it reads that kernel's
// output.  pdl_release lets the next such kernel be scheduled once every CTA
// of this one has started.  Both are no-ops for plain launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Packed FP32x2 a * b + c, a * b and a + b, round-to-nearest per lane (each
// lane is bitwise the scalar __fmaf_rn / __fmul_rn / __fadd_rn).
__device__ __forceinline__ unsigned long long fma2_rn(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long mul2_rn(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ unsigned long long add2_rn(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Butterfly (xor) sum: every lane ends with the bitwise-identical total,
// because each level adds the same two operands in either order.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Index of cell (x, y), 0 <= x, y < 2^ORDER, along the Hilbert curve of that
// order.  Classic iterative form: from the top level down, the quadrant of
// (x, y) gives two bits of the index (quadrants visited in the order (0,0),
// (0,1), (1,1), (1,0)), and (x, y) is carried into that quadrant's own frame -
// the first quadrant transposed, the last one reflected through the
// anti-diagonal - so that the curve of the level below enters and leaves where
// the level above needs it.  Consecutive indices are edge-adjacent cells (a
// Morton order jumps at every quadrant edge), so runs of consecutive points
// stay compact.
template <int ORDER>
__device__ __forceinline__ uint32_t hilbert_index(uint32_t x, uint32_t y) {
    uint32_t d = 0;
#pragma unroll
    for (int lev = ORDER - 1; lev >= 0; --lev) {
        const uint32_t s = 1u << lev;
        const uint32_t rx = (x >> lev) & 1u, ry = (y >> lev) & 1u;
        d += s * s * ((3u * rx) ^ ry);
        x &= s - 1;
        y &= s - 1;
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - x;
                y = s - 1 - y;
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
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

// Bitonic sort of C = THREADS * R distinct keys held in registers, thread t
// owning positions t R .. t R + R - 1 (all THREADS threads of the block call
// it).  Partners closer than R sit in the same thread, closer than 32 R in the
// same warp (shuffles); farther ones are exchanged through shared memory `x`
// (C keys).  Element i of a pair (i, i ^ j) inside a run sorted upwards
// ((i & k) == 0) keeps the smaller key when it is the lower index.
template <typename T, int R, int THREADS>
__device__ __forceinline__ void bitonic_sort_regs(T (&v)[R], T *x) {
    constexpr int C = THREADS * R;
    const int t = threadIdx.x;
#pragma unroll 1
    for (int k = 2; k <= C; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j >= R; j >>= 1) {
            if (j >= 32 * R) {
#pragma unroll
                for (int r = 0; r < R; ++r) x[t * R + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = t * R + r;
                    const T b = x[i ^ j];
                    const bool keep_min = ((i & k) == 0) == (i < (i ^ j));
                    v[r] = keep_min ? (v[r] < b ? v[r] : b) : (v[r] > b ? v[r] : b);
                }
                __syncthreads();
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = t * R + r;
                    const T b = __shfl_xor_sync(0xffffffffu, v[r], j / R);
                    const bool keep_min = ((i & k) == 0) == (i < (i ^ j));
                    v[r] = keep_min ? (v[r] < b ? v[r] : b) : (v[r] > b ? v[r] : b);
                }
            }
        }
        // partners inside the thread: compile-time register indices
#pragma unroll
        for (int j = R / 2; j >= 1; j >>= 1) {
            if (j > (k >> 1)) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r & j) continue;
                const int i = t * R + r;
                const T a = v[r], b = v[r | j];
                if ((a > b) == ((i & k) == 0)) {
                    v[r] = b;
                    v[r | j] = a;
                }
            }
        }
    }
}

}  // namespace retina
