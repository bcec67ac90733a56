// Throughput probe of the FP32 FMA pipe and the MUFU (SFU) ex2 pipe, the two
// units the retina kernels are bound by.  One saturating launch (8 CTAs of
// 256 threads per SM), eight independent dependency chains per thread; the
// caller times it with CUDA events and divides the reported operation count
// by the time.  Not part of the paper: it measures the roofline's peaks.
#include "internal.cuh"

namespace retina {

constexpr int PROBE_THREADS = 256, PROBE_CTAS_PER_SM = 8, PROBE_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) alu_probe_kernel(int iters, float *__restrict__ sink) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = 0.5f + 1e-3f * i + 1e-7f * (float)threadIdx.x;
    if (KIND == 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = __fmaf_rn(a[i], 0.99990f, 1.0e-4f);
        }
    } else if (KIND == 1) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = ex2_mufu(-a[i]);
        }
    } else {
        unsigned long long x[PROBE_CHAINS / 2];
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS / 2; ++i)
            x[i] = ((unsigned long long)__float_as_uint(a[2 * i + 1]) << 32) | __float_as_uint(a[2 * i]);
        const unsigned long long m = ((unsigned long long)__float_as_uint(0.99990f) << 32) | __float_as_uint(0.99990f);
        const unsigned long long c = ((unsigned long long)__float_as_uint(1.0e-4f) << 32) | __float_as_uint(1.0e-4f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS / 2; ++i)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(m), "l"(c));
        }
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS / 2; ++i) {
            a[2 * i] = __uint_as_float((unsigned)(x[i] & 0xffffffffull));
            a[2 * i + 1] = __uint_as_float((unsigned)(x[i] >> 32));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    sink[gid] = s;
}

}  // namespace retina

using namespace retina;

extern "C" {

int64_t retina_alu_probe_sink_floats(void) { return (int64_t)sm_count() * PROBE_CTAS_PER_SM * PROBE_THREADS; }

int retina_alu_probe(int32_t kind, int32_t iters, float *sink, double *ops, void *stream) {
    if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 20) || !sink || !ops) return RETINA_EINVAL;
    const int blocks = sm_count() * PROBE_CTAS_PER_SM;
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == 0)
        alu_probe_kernel<0><<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
    else if (kind == 1)
        alu_probe_kernel<1><<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
    else
        alu_probe_kernel<2><<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
    count_launches(1);
    *ops = (double)blocks * PROBE_THREADS * (double)iters * PROBE_CHAINS;
    return cudaGetLastError() == cudaSuccess ? RETINA_OK : RETINA_ECUDA;
}

}  // extern "C"
