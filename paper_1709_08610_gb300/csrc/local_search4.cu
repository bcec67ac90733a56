// Algorithm 1 with the truncated Newton update of Section 3 for a
// four-parameter straight track theta = (x0, y0, t_x, t_y) at a reference
// plane z_ref: the track crosses the layer z at (x0 + t_x w, y0 + t_y w),
// w = z - z_ref, so it need not pass through the origin (a vertex displaced
// along or across the beam is representable).
//
// Residual r = (x - x0 - t_x w, y - y0 - t_y w), J = -dr/dtheta =
// [[1, 0, w, 0], [0, 1, 0, w]], e = exp(-|r|^2 / sigma^2), k = 1 / sigma^2:
//   grad R = 2k sum e J^T r,  J^T r = (r0, r1, w r0, w r1)
//   Hess R = 4k^2 sum e (J^T r)(J^T r)^T - 2k sum e J^T J
// Each lane accumulates 16 sums over a stride of the event's hits (z below
// stands for w):
//   S0 e, S1 e r0, S2 e r1, S3 e z r0, S4 e z r1,
//   S5 e r0^2, S6 e r0 r1, S7 e r1^2, S8 e z r0^2, S9 e z r0 r1, S10 e z r1^2,
//   S11 e z^2 r0^2, S12 e z^2 r0 r1, S13 e z^2 r1^2, S14 e z, S15 e z^2
// then a butterfly reduction leaves the totals in every lane, so every
// decision is warp-uniform.  One warp per seed, hits staged in shared memory
// (the rest read through L1); no block skipping.
#include "internal.cuh"

namespace retina {

struct Ls4Params {
    int q;
    float kk[RETINA_MAX_Q];  // log2(e) / sigma_j^2
    float k[RETINA_MAX_Q];   // 1 / sigma_j^2
    float c1;
    int max_halvings;
    float scale[4];
    float inv_scale[4];
    float cap;
    float zref;
};

// Symmetric 4 x 4 Hessian from the sums: H[a][b].
__device__ __forceinline__ void hess4_from_sums(const float *S, float k, float H[4][4]) {
    const float k4 = 4.f * k * k, k2 = 2.f * k;
    // e (J^T r)_a (J^T r)_b
    const float O[4][4] = {{S[5], S[6], S[8], S[9]},
                           {S[6], S[7], S[9], S[10]},
                           {S[8], S[9], S[11], S[12]},
                           {S[9], S[10], S[12], S[13]}};
    // e (J^T J)_ab
    const float JJ[4][4] = {{S[0], 0.f, S[14], 0.f}, {0.f, S[0], 0.f, S[14]}, {S[14], 0.f, S[15], 0.f},
                            {0.f, S[14], 0.f, S[15]}};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) H[a][b] = k4 * O[a][b] - k2 * JJ[a][b];
}

// Newton-CG direction for maximising R in four dimensions (Nocedal & Wright,
// Algorithm 7.1) in the variables scaled by the parameters' units D =
// diag(scale): CG on (D B D) y = D g, B = -H, from y = 0, forcing tolerance
// min(1/2, sqrt|D g|) |D g|, at most 4 iterations, non-positive curvature
// gives y = D g at the first iteration and the current iterate after;
// p = D y.  The scaled g and B are further scaled by one power of two
// (exact; the direction is unchanged) so that no square underflows.
__device__ __forceinline__ void newton_cg4(const float g_in[4], const float H[4][4], const float scale[4],
                                           float p[4]) {
    float g[4];
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        g[a] = g_in[a] * scale[a];
        m = fmaxf(m, fabsf(g[a]));
    }
    if (m == 0.f || !isfinite(m)) {
#pragma unroll
        for (int a = 0; a < 4; ++a) p[a] = g[a] * scale[a];
        return;
    }
    int ex;
    frexpf(m, &ex);
    if (ex & 1) ++ex;
    const float c = ldexpf(1.f, -ex);
    float sg[4], B[4][4], gn2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        sg[a] = g[a] * c;
        gn2 += sg[a] * sg[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) B[a][b] = -(scale[a] * H[a][b] * scale[b]) * c;
    }
    const float gn_s = sqrtf(gn2);
    const float sqrt_gn = sqrtf(gn_s) * ldexpf(1.f, ex / 2);
    const float eps_s = fminf(0.5f, sqrt_gn) * gn_s;
    float z[4] = {0.f, 0.f, 0.f, 0.f}, r[4], d[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        r[a] = -sg[a];
        d[a] = sg[a];
    }
    for (int it = 0; it < 4; ++it) {
        float Bd[4], dBd = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            Bd[a] = B[a][0] * d[0] + B[a][1] * d[1] + B[a][2] * d[2] + B[a][3] * d[3];
            dBd += d[a] * Bd[a];
        }
        if (dBd <= 0.f) {
#pragma unroll
            for (int a = 0; a < 4; ++a) p[a] = (it == 0 ? g[a] : z[a]) * scale[a];
            return;
        }
        float rr = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) rr += r[a] * r[a];
        const float alpha = rr / dBd;
        float rn[4], rnn2 = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            z[a] += alpha * d[a];
            rn[a] = r[a] + alpha * Bd[a];
            rnn2 += rn[a] * rn[a];
        }
        if (sqrtf(rnn2) < eps_s) break;
        const float beta = rnn2 / rr;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            d[a] = -rn[a] + beta * d[a];
            r[a] = rn[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) p[a] = z[a] * scale[a];
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
local_search4_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, int n_seeds,
                     const int32_t *__restrict__ seed_count, const float *__restrict__ seeds, Ls4Params prm,
                     int smem_hits, float *__restrict__ theta_out, float *__restrict__ R_out,
                     uint8_t *__restrict__ status) {
    extern __shared__ float4 sh[];
    const int e = blockIdx.y;
    // seeds [count, n_seeds) of the event are not searched; a CTA with none
    // of its seeds below the count leaves before staging (uniformly)
    int count = n_seeds;
    if (seed_count) {
        const int c = seed_count[e];
        count = c < 0 ? 0 : (c < n_seeds ? c : n_seeds);
    }
    if (blockIdx.x * WARPS >= count) return;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int H = (int)(he - hb);
    const float4 *gh = hits + hb;
    const int n_staged = H < smem_hits ? H : smem_hits;
    for (int i = threadIdx.x; i < n_staged; i += blockDim.x) sh[i] = __ldg(gh + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (s >= count) return;  // after the only barrier
    const int64_t o = (int64_t)e * n_seeds + s;
    float th[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) th[a] = seeds[4 * o + a];
    bool failed = false;
    float Rfin = 0.f;
    for (int j = 0; j < prm.q; ++j) {
        const float kk = prm.kk[j], k = prm.k[j];
        float S[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) S[i] = 0.f;
        for (int i = lane; i < H; i += 32) {
            const float4 h = i < n_staged ? sh[i] : __ldg(gh + i);
            // x - t_x w rounded once (about x0 + r0), then the exact
            // difference to x0: the error is a rounding of |x0|, not of |x|
            const float w = h.z - prm.zref;
            const float r0 = __fsub_rn(__fmaf_rn(-th[2], w, h.x), th[0]);
            const float r1 = __fsub_rn(__fmaf_rn(-th[3], w, h.y), th[1]);
            const float ev = ex2_mufu(-__fmaf_rn(r0, r0, r1 * r1) * kk);
            const float ez = ev * w, ez2 = ez * w;
            S[0] += ev;
            S[1] = __fmaf_rn(ev, r0, S[1]);
            S[2] = __fmaf_rn(ev, r1, S[2]);
            S[3] = __fmaf_rn(ez, r0, S[3]);
            S[4] = __fmaf_rn(ez, r1, S[4]);
            const float er0 = ev * r0, er1 = ev * r1, ezr0 = ez * r0, ezr1 = ez * r1, ez2r0 = ez2 * r0;
            S[5] = __fmaf_rn(er0, r0, S[5]);
            S[6] = __fmaf_rn(er0, r1, S[6]);
            S[7] = __fmaf_rn(er1, r1, S[7]);
            S[8] = __fmaf_rn(ezr0, r0, S[8]);
            S[9] = __fmaf_rn(ezr0, r1, S[9]);
            S[10] = __fmaf_rn(ezr1, r1, S[10]);
            S[11] = __fmaf_rn(ez2r0, r0, S[11]);
            S[12] = __fmaf_rn(ez2r0, r1, S[12]);
            S[13] = __fmaf_rn(ez2 * r1, r1, S[13]);
            S[14] += ez;
            S[15] += ez2;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) S[i] = warp_sum(S[i]);
        const float R = S[0];
        const float k2 = 2.f * k;
        const float g[4] = {k2 * S[1], k2 * S[2], k2 * S[3], k2 * S[4]};
        float Hm[4][4];
        hess4_from_sums(S, k, Hm);
        float p[4];
        newton_cg4(g, Hm, prm.scale, p);
        float cells = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) cells = fmaxf(cells, fabsf(p[a]) * prm.inv_scale[a]);
        if (cells > prm.cap) {
            const float sc = prm.cap / cells;
#pragma unroll
            for (int a = 0; a < 4; ++a) p[a] *= sc;
        }
        const float slope = g[0] * p[0] + g[1] * p[1] + g[2] * p[2] + g[3] * p[3];
        float t = 1.f;
        bool pending = true;
        Rfin = R;
        for (int hv = 0; hv <= prm.max_halvings && pending; ++hv) {
            float tr[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) tr[a] = __fmaf_rn(t, p[a], th[a]);
            float Rt = 0.f;
            for (int i = lane; i < H; i += 32) {
                const float4 h = i < n_staged ? sh[i] : __ldg(gh + i);
                const float w = h.z - prm.zref;
                const float r0 = __fsub_rn(__fmaf_rn(-tr[2], w, h.x), tr[0]);
                const float r1 = __fsub_rn(__fmaf_rn(-tr[3], w, h.y), tr[1]);
                Rt += ex2_mufu(-__fmaf_rn(r0, r0, r1 * r1) * kk);
            }
            Rt = warp_sum(Rt);
            if (Rt >= R + prm.c1 * t * slope) {
#pragma unroll
                for (int a = 0; a < 4; ++a) th[a] = tr[a];
                Rfin = Rt;
                pending = false;
            } else {
                t *= 0.5f;
            }
        }
        if (pending) failed = true;
    }
    if (lane != 0) return;
    bool fin = isfinite(Rfin);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        theta_out[4 * o + a] = th[a];
        fin = fin && isfinite(th[a]);
    }
    R_out[o] = Rfin;
    status[o] = fin ? (failed ? 1 : 0) : 3;
}

cudaError_t launch_local_search4(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events,
                                 const float *seeds, int n_seeds, const int32_t *seed_count, const retina_ls4_opts *o,
                                 float *theta_out, float *R_out, uint8_t *status, int smem_hits, cudaStream_t st) {
    Ls4Params prm;
    prm.q = o->q;
    for (int j = 0; j < RETINA_MAX_Q; ++j) {
        const double sg = j < o->q ? (double)o->sigma[j] : 1.0;
        prm.kk[j] = (float)(kLog2e / (sg * sg));
        prm.k[j] = (float)(1.0 / (sg * sg));
    }
    prm.c1 = o->c1;
    prm.max_halvings = o->max_halvings;
    for (int a = 0; a < 4; ++a) {
        prm.scale[a] = o->scale[a];
        prm.inv_scale[a] = (float)(1.0 / (double)o->scale[a]);
    }
    prm.cap = o->step_cap;
    prm.zref = o->zref;
    if (smem_hits < 0) smem_hits = 0;
    if (smem_hits > 12288) smem_hits = 12288;
    constexpr int WARPS = 8;
    const size_t smem = (size_t)smem_hits * sizeof(float4);
    cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(local_search4_kernel<WARPS>), smem);
    if (aerr != cudaSuccess) return aerr;
    dim3 grid((n_seeds + WARPS - 1) / WARPS, n_events);
    local_search4_kernel<WARPS><<<grid, WARPS * 32, smem, st>>>(hits, n_hits, off, n_seeds, seed_count, seeds, prm,
                                                              smem_hits, theta_out, R_out, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
