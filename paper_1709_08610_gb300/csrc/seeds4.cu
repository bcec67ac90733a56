// Starting points of the four-parameter search from pairs of hits
// (retina_pair_seeds4; the paper has no four-parameter search and leaves the
// prior P_theta of Algorithm 1 open).  Tracks come from the beam line: a pair
// of hits of one track on two layers spans a line that passes close to the z
// axis inside the luminous region, a pair from two tracks rarely does.
//
// One CTA per event.  For each layer pair, the hits of the two layers are
// listed in increasing index order (ordered compaction), then the pairs are
// tested in (i, j) order, a CTA-wide tile at a time, and the kept ones are
// written in that order (ordered compaction again), so the seed list is a
// deterministic function of the event.  Every decision is taken in float32
// with one rounding per operation (explicit _rn intrinsics, no contraction),
// in the order the definition writes it.
#include "internal.cuh"

namespace retina {

constexpr int PS_THREADS = 256;

struct PairSeedParams {
    float za[RETINA_MAX_LAYER_PAIRS], zb[RETINA_MAX_LAYER_PAIRS];
    int n_pairs;
    float dz_tol, d_max, zc_lo, zc_hi, zref;
    int K;
};

// Exclusive position of this thread's flag among the CTA's flags (thread
// order), and the CTA total.  All threads call it.
__device__ __forceinline__ int cta_rank(bool flag, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < PS_THREADS / 32; ++w) {
        const int v = warp_tot[w];
        before += w < warp ? v : 0;
        total += v;
    }
    __syncthreads();  // warp_tot is rewritten by the next call
    return before + __popc(m & ((1u << lane) - 1u));
}

// List the indices (relative to the event) of the event's hits with
// |z - z_layer| <= tol, in increasing order; returns how many (at most cap
// are stored, the count is not clamped).  All threads call it; the list is
// complete for every thread when it returns.
__device__ int list_layer(const float4 *__restrict__ gh, int H, float z_layer, float tol, int *idx, int cap,
                          int *warp_tot) {
    int n = 0;
    for (int k0 = 0; k0 < H; k0 += PS_THREADS) {
        const int k = k0 + threadIdx.x;
        const bool in = k < H && fabsf(__fsub_rn(__ldg(gh + k).z, z_layer)) <= tol;
        int total;
        const int pos = cta_rank(in, warp_tot, total);
        if (in && n + pos < cap) idx[n + pos] = k;
        n += total;
    }
    __syncthreads();  // the last window's entries are read by other threads next
    return n;
}

__global__ void __launch_bounds__(PS_THREADS)
pair_seeds4_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, PairSeedParams prm,
                   float *__restrict__ seeds, int32_t *__restrict__ n_seeds) {
    __shared__ int idx_a[RETINA_PAIR_LAYER_CAP], idx_b[RETINA_PAIR_LAYER_CAP];
    __shared__ int warp_tot[PS_THREADS / 32];
    const int e = blockIdx.x;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int H = (int)(he - hb);
    const float4 *gh = hits + hb;
    const float dm2 = __fmul_rn(prm.d_max, prm.d_max);
    float *out = seeds + (int64_t)e * prm.K * 4;
    int count = 0;
    bool overflow = false;
    for (int p = 0; p < prm.n_pairs; ++p) {
        int na = list_layer(gh, H, prm.za[p], prm.dz_tol, idx_a, RETINA_PAIR_LAYER_CAP, warp_tot);
        int nb = list_layer(gh, H, prm.zb[p], prm.dz_tol, idx_b, RETINA_PAIR_LAYER_CAP, warp_tot);
        overflow |= na > RETINA_PAIR_LAYER_CAP || nb > RETINA_PAIR_LAYER_CAP;
        na = na < RETINA_PAIR_LAYER_CAP ? na : RETINA_PAIR_LAYER_CAP;
        nb = nb < RETINA_PAIR_LAYER_CAP ? nb : RETINA_PAIR_LAYER_CAP;
        const int64_t n_pair = (int64_t)na * nb;
        for (int64_t q0 = 0; q0 < n_pair; q0 += PS_THREADS) {
            const int64_t q = q0 + threadIdx.x;
            bool keep = false;
            float s0 = 0.f, s1 = 0.f, tx = 0.f, ty = 0.f;
            if (q < n_pair) {
                const float4 hi = __ldg(gh + idx_a[q / nb]), hj = __ldg(gh + idx_b[q % nb]);
                const float dz = __fsub_rn(hj.z, hi.z);
                tx = __fdiv_rn(__fsub_rn(hj.x, hi.x), dz);
                ty = __fdiv_rn(__fsub_rn(hj.y, hi.y), dz);
                const float tt = __fadd_rn(__fmul_rn(tx, tx), __fmul_rn(ty, ty));
                if (tt > 0.f) {
                    const float c = __fsub_rn(__fmul_rn(hi.x, ty), __fmul_rn(hi.y, tx));
                    if (__fmul_rn(c, c) <= __fmul_rn(dm2, tt)) {
                        const float u = __fadd_rn(__fmul_rn(hi.x, tx), __fmul_rn(hi.y, ty));
                        const float zc = __fsub_rn(hi.z, __fdiv_rn(u, tt));
                        if (zc >= prm.zc_lo && zc <= prm.zc_hi) {
                            keep = true;
                            const float w = __fsub_rn(prm.zref, hi.z);
                            s0 = __fadd_rn(hi.x, __fmul_rn(tx, w));
                            s1 = __fadd_rn(hi.y, __fmul_rn(ty, w));
                        }
                    }
                }
            }
            int total;
            const int pos = count + cta_rank(keep, warp_tot, total);
            if (keep && pos < prm.K) {
                out[4 * pos] = s0;
                out[4 * pos + 1] = s1;
                out[4 * pos + 2] = tx;
                out[4 * pos + 3] = ty;
            }
            count += total;
        }
    }
    // a layer with more hits than the lists hold: the pairing was incomplete
    if (threadIdx.x == 0) n_seeds[e] = overflow ? -1 : count;
}

cudaError_t launch_pair_seeds4(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events,
                               const float *layer_z, int n_pairs, float dz_tol, float d_max, float zc_lo, float zc_hi,
                               float zref, float *seeds, int32_t *n_seeds, int K, cudaStream_t st) {
    PairSeedParams prm{};
    for (int p = 0; p < n_pairs; ++p) {
        prm.za[p] = layer_z[2 * p];
        prm.zb[p] = layer_z[2 * p + 1];
    }
    prm.n_pairs = n_pairs;
    prm.dz_tol = dz_tol;
    prm.d_max = d_max;
    prm.zc_lo = zc_lo;
    prm.zc_hi = zc_hi;
    prm.zref = zref;
    prm.K = K;
    pair_seeds4_kernel<<<n_events, PS_THREADS, 0, st>>>(hits, n_hits, off, prm, seeds, n_seeds);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
