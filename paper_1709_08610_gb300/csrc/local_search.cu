// Multistart local search (Algorithm 1) with the truncated Newton update and
// annealed bandwidth of Section 3, plus point-wise R / grad R / Hess R.
//
// Layout: one warp owns P seeds of one event; its 32 lanes stride over the
// event's hits (staged once per CTA in shared memory, float4 per hit; hits
// beyond the staged capacity are read through L1/L2), each lane accumulating
// the sums of Eq. 1 and its derivatives for all P seeds, then a xor-butterfly
// reduction leaves bitwise-identical totals in every lane.  Every decision
// (CG branch, step cap, Armijo test) is therefore warp-uniform: no lane ever
// diverges from its warp, and seeds that finished their line search idle
// under a uniform predicate.
//
// Sums per pair, with e = exp(-|r|^2 / sigma^2), k = 1 / sigma^2:
//   slope model (J = z I):     S = [e, e z rx, e z ry, e z^2 rx^2, e z^2 rx ry, e z^2 ry^2, e z^2]
//     grad = 2k (S1, S2);  H = 4k^2 [S3 S4; S4 S5] - 2k S6 I
//   2D toy (J = [x, 1]):       S = [e, e r x, e r, e r^2 x^2, e r^2 x, e r^2, e x^2, e x]
//     grad = 2k (S1, S2);  H = 4k^2 [S3 S4; S4 S5] - 2k [S6 S7; S7 S0]
#include "internal.cuh"

namespace retina {

constexpr int LS_WARPS = 8;

template <int MODEL>
struct Model {
    static constexpr int NS = (MODEL == RETINA_VELO_SLOPES) ? 7 : 8;
};

// One pair's contribution to the RGH sums (MUFU ex2 + FMA-pipe arithmetic).
template <int MODEL>
__device__ __forceinline__ void pair_rgh(const float4 h, float t0, float t1, float kk, float *S) {
    if (MODEL == RETINA_VELO_SLOPES) {
        const float rx = __fmaf_rn(-t0, h.z, h.x);
        const float ry = __fmaf_rn(-t1, h.z, h.y);
        const float s2 = __fmaf_rn(rx, rx, ry * ry);
        const float e = ex2_mufu(-s2 * kk);
        const float ez = e * h.z;
        const float ez2 = ez * h.z;
        const float ez2rx = ez2 * rx;
        S[0] += e;
        S[1] = __fmaf_rn(ez, rx, S[1]);
        S[2] = __fmaf_rn(ez, ry, S[2]);
        S[3] = __fmaf_rn(ez2rx, rx, S[3]);
        S[4] = __fmaf_rn(ez2rx, ry, S[4]);
        S[5] = __fmaf_rn(ez2 * ry, ry, S[5]);
        S[6] += ez2;
    } else {
        const float r = __fmaf_rn(-t0, h.x, h.y) - t1;
        const float e = ex2_mufu(-(r * r) * kk);
        const float er = e * r;
        const float erx = er * h.x;
        const float ex = e * h.x;
        S[0] += e;
        S[1] += erx;
        S[2] += er;
        S[3] = __fmaf_rn(erx * r, h.x, S[3]);
        S[4] = __fmaf_rn(erx, r, S[4]);
        S[5] = __fmaf_rn(er, r, S[5]);
        S[6] = __fmaf_rn(ex, h.x, S[6]);
        S[7] += ex;
    }
}

template <int MODEL>
__device__ __forceinline__ float pair_r(const float4 h, float t0, float t1, float kk) {
    if (MODEL == RETINA_VELO_SLOPES) {
        const float rx = __fmaf_rn(-t0, h.z, h.x);
        const float ry = __fmaf_rn(-t1, h.z, h.y);
        return ex2_mufu(-__fmaf_rn(rx, rx, ry * ry) * kk);
    } else {
        const float r = __fmaf_rn(-t0, h.x, h.y) - t1;
        return ex2_mufu(-(r * r) * kk);
    }
}

template <int MODEL>
__device__ __forceinline__ void sums_to_rgh(const float *S, float k, float &R, float &g0, float &g1, float &H00,
                                            float &H01, float &H11) {
    const float k2 = 2.f * k, k4 = 4.f * k * k;
    R = S[0];
    g0 = k2 * S[1];
    g1 = k2 * S[2];
    if (MODEL == RETINA_VELO_SLOPES) {
        H00 = k4 * S[3] - k2 * S[6];
        H01 = k4 * S[4];
        H11 = k4 * S[5] - k2 * S[6];
    } else {
        H00 = k4 * S[3] - k2 * S[6];
        H01 = k4 * S[4] - k2 * S[7];
        H11 = k4 * S[5] - k2 * S[0];
    }
}

__device__ __forceinline__ float4 load_hit(const float4 *__restrict__ sh, const float4 *__restrict__ gh, int k,
                                           int n_staged) {
    return k < n_staged ? sh[k] : __ldg(gh + k);
}

// Newton-CG direction for maximising R (minimising -R: gradient -g,
// Hessian B = -H), from p = 0, forcing tolerance min(1/2, sqrt|g|)|g|,
// at most two iterations; non-positive curvature of B along the CG
// direction returns g (first iteration) or the current iterate.  g and B are
// scaled by a power of two so that no intermediate underflows; the scaling is
// exact and leaves the direction unchanged.
__device__ __forceinline__ void newton_cg(float g0, float g1, float H00, float H01, float H11, float &p0,
                                          float &p1) {
    const float m = fmaxf(fabsf(g0), fabsf(g1));
    if (m == 0.f) {  // d = g = 0 -> zero curvature at the first iteration -> p = g
        p0 = g0;
        p1 = g1;
        return;
    }
    if (!isfinite(m)) {
        p0 = g0;
        p1 = g1;
        return;
    }
    int ex;
    frexpf(m, &ex);
    if (ex & 1) ++ex;  // even, so that sqrt of the scale is exact
    const float c = ldexpf(1.f, -ex);
    const float sg0 = g0 * c, sg1 = g1 * c;
    const float B00 = -H00 * c, B01 = -H01 * c, B11 = -H11 * c;
    const float gn_s = sqrtf(sg0 * sg0 + sg1 * sg1);  // |g| * c
    const float sqrt_gn = sqrtf(gn_s) * ldexpf(1.f, ex / 2);
    const float eps_s = fminf(0.5f, sqrt_gn) * gn_s;  // eps * c
    float z0 = 0.f, z1 = 0.f, r0 = -sg0, r1 = -sg1, d0 = sg0, d1 = sg1;
    for (int it = 0; it < 2; ++it) {
        const float Bd0 = B00 * d0 + B01 * d1;
        const float Bd1 = B01 * d0 + B11 * d1;
        const float dBd = d0 * Bd0 + d1 * Bd1;
        if (dBd <= 0.f) {
            if (it == 0) {
                p0 = g0;
                p1 = g1;
            } else {
                p0 = z0;
                p1 = z1;
            }
            return;
        }
        const float rr = r0 * r0 + r1 * r1;
        const float alpha = rr / dBd;
        z0 += alpha * d0;
        z1 += alpha * d1;
        const float rn0 = r0 + alpha * Bd0, rn1 = r1 + alpha * Bd1;
        const float rnn2 = rn0 * rn0 + rn1 * rn1;
        if (sqrtf(rnn2) < eps_s) break;
        const float beta = rnn2 / rr;
        d0 = -rn0 + beta * d0;
        d1 = -rn1 + beta * d1;
        r0 = rn0;
        r1 = rn1;
    }
    p0 = z0;
    p1 = z1;
}

struct LsParams {
    int q;
    float kk[RETINA_MAX_Q];  // log2(e) / sigma_j^2
    float k[RETINA_MAX_Q];   // 1 / sigma_j^2
    float c1;
    int max_halvings;
    float cap;
    GridDev box;
};

template <int MODEL, int P>
__global__ void __launch_bounds__(LS_WARPS * 32)
local_search_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, int n_seeds,
                    const float *__restrict__ seeds, LsParams prm, int smem_hits, float *__restrict__ theta_out,
                    float *__restrict__ R_out, uint8_t *__restrict__ status, uint8_t *__restrict__ n_evals) {
    extern __shared__ float4 sh[];
    constexpr int NS = Model<MODEL>::NS;
    const int e = blockIdx.y;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int H = (int)(he - hb);
    const float4 *gh = hits + hb;
    const int n_staged = H < smem_hits ? H : smem_hits;
    for (int k = threadIdx.x; k < n_staged; k += blockDim.x) sh[k] = __ldg(gh + k);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s_first = (blockIdx.x * LS_WARPS + warp) * P;
    if (s_first >= n_seeds) return;

    float th0[P], th1[P];
    int evals[P];
    bool live[P], failed[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int s = s_first + p;
        live[p] = s < n_seeds;
        const int64_t o = ((int64_t)e * n_seeds + (live[p] ? s : s_first)) * 2;
        th0[p] = seeds[o];
        th1[p] = seeds[o + 1];
        failed[p] = false;
        evals[p] = 1;  // the final response pass
    }

    for (int j = 0; j < prm.q; ++j) {
        const float kk = prm.kk[j], k = prm.k[j];
        // (R, g, H) at the current points
        float S[P][NS];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < NS; ++i) S[p][i] = 0.f;
        for (int kh = lane; kh < H; kh += 32) {
            const float4 h = load_hit(sh, gh, kh, n_staged);
#pragma unroll
            for (int p = 0; p < P; ++p) pair_rgh<MODEL>(h, th0[p], th1[p], kk, S[p]);
        }
        float R[P], g0[P], g1[P], pp0[P], pp1[P], slope[P], t[P];
        bool pending[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int i = 0; i < NS; ++i) S[p][i] = warp_sum(S[p][i]);
            float H00, H01, H11;
            sums_to_rgh<MODEL>(S[p], k, R[p], g0[p], g1[p], H00, H01, H11);
            newton_cg(g0[p], g1[p], H00, H01, H11, pp0[p], pp1[p]);
            const float cells = fmaxf(fabsf(pp0[p]) / prm.box.step0, fabsf(pp1[p]) / prm.box.step1);
            if (cells > prm.cap) {
                const float sc = prm.cap / cells;
                pp0[p] *= sc;
                pp1[p] *= sc;
            }
            slope[p] = g0[p] * pp0[p] + g1[p] * pp1[p];
            t[p] = 1.f;
            pending[p] = live[p];
        }
        // backtracking line search, all pending seeds of the warp together
        for (int hv = 0; hv <= prm.max_halvings; ++hv) {
            bool any = false;
#pragma unroll
            for (int p = 0; p < P; ++p) any |= pending[p];
            if (!any) break;
            float tr0[P], tr1[P], Rt[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                tr0[p] = __fmaf_rn(t[p], pp0[p], th0[p]);
                tr1[p] = __fmaf_rn(t[p], pp1[p], th1[p]);
                Rt[p] = 0.f;
            }
            for (int kh = lane; kh < H; kh += 32) {
                const float4 h = load_hit(sh, gh, kh, n_staged);
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (pending[p]) Rt[p] += pair_r<MODEL>(h, tr0[p], tr1[p], kk);
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (!pending[p]) continue;
                ++evals[p];
                const float rt = warp_sum(Rt[p]);
                if (rt >= R[p] + prm.c1 * t[p] * slope[p]) {
                    th0[p] = tr0[p];
                    th1[p] = tr1[p];
                    pending[p] = false;
                } else {
                    t[p] *= 0.5f;
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (pending[p]) failed[p] = true;
    }

    // final response at the last bandwidth
    const float kkq = prm.kk[prm.q - 1];
    float Rf[P];
#pragma unroll
    for (int p = 0; p < P; ++p) Rf[p] = 0.f;
    for (int kh = lane; kh < H; kh += 32) {
        const float4 h = load_hit(sh, gh, kh, n_staged);
#pragma unroll
        for (int p = 0; p < P; ++p) Rf[p] += pair_r<MODEL>(h, th0[p], th1[p], kkq);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float rf = warp_sum(Rf[p]);
        if (!live[p] || lane != 0) continue;
        const int64_t o = (int64_t)e * n_seeds + s_first + p;
        uint8_t st;
        const float hi0 = prm.box.lo0 + (float)prm.box.n0 * prm.box.step0;
        const float hi1 = prm.box.lo1 + (float)prm.box.n1 * prm.box.step1;
        if (!(isfinite(th0[p]) && isfinite(th1[p]) && isfinite(rf)))
            st = 3;
        else if (!(th0[p] >= prm.box.lo0 && th0[p] < hi0 && th1[p] >= prm.box.lo1 && th1[p] < hi1))
            st = 2;
        else
            st = failed[p] ? 1 : 0;
        theta_out[2 * o] = th0[p];
        theta_out[2 * o + 1] = th1[p];
        R_out[o] = rf;
        status[o] = st;
        if (n_evals) n_evals[o] = (uint8_t)(evals[p] < 255 ? evals[p] : 255);
    }
}

// R (and optionally grad R, Hess R) at arbitrary points: one warp per point.
template <int MODEL>
__global__ void __launch_bounds__(256)
response_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off, int n_points,
                const float *__restrict__ theta, float kk, float k, int want_derivs, float *__restrict__ out) {
    constexpr int NS = Model<MODEL>::NS;
    const int e = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int pt = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pt >= n_points) return;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int H = (int)(he - hb);
    const int64_t o = (int64_t)e * n_points + pt;
    const float t0 = theta[2 * o], t1 = theta[2 * o + 1];
    float S[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = 0.f;
    for (int kh = lane; kh < H; kh += 32) {
        const float4 h = __ldg(hits + hb + kh);
        if (want_derivs)
            pair_rgh<MODEL>(h, t0, t1, kk, S);
        else
            S[0] += pair_r<MODEL>(h, t0, t1, kk);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = warp_sum(S[i]);
    if (lane != 0) return;
    float R, g0, g1, H00, H01, H11;
    sums_to_rgh<MODEL>(S, k, R, g0, g1, H00, H01, H11);
    float *dst = out + o * 6;
    dst[0] = R;
    if (want_derivs) {
        dst[1] = g0;
        dst[2] = g1;
        dst[3] = H00;
        dst[4] = H01;
        dst[5] = H11;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <int MODEL, int P>
static cudaError_t launch_ls_t(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int n_seeds,
                               const float *seeds,
                               const LsParams &prm, int smem_hits, float *theta_out, float *R_out, uint8_t *status,
                               uint8_t *n_evals, cudaStream_t st) {
    const size_t smem = (size_t)smem_hits * sizeof(float4);
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(local_search_kernel<MODEL, P>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    const int per_block = LS_WARPS * P;
    dim3 grid((n_seeds + per_block - 1) / per_block, n_events);
    local_search_kernel<MODEL, P><<<grid, LS_WARPS * 32, smem, st>>>(hits, n_hits, off, n_seeds, seeds, prm, smem_hits,
                                                                      theta_out, R_out, status, n_evals);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_search(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                                const float *seeds,
                                int n_seeds, const retina_ls_opts *o, const retina_grid *box, float *theta_out,
                                float *R_out, uint8_t *status, uint8_t *n_evals, int seeds_per_warp, int smem_hits,
                                cudaStream_t st) {
    LsParams prm;
    prm.q = o->q;
    for (int j = 0; j < RETINA_MAX_Q; ++j) {
        const double s = j < o->q ? (double)o->sigma[j] : 1.0;
        prm.kk[j] = (float)(kLog2e / (s * s));
        prm.k[j] = (float)(1.0 / (s * s));
    }
    prm.c1 = o->c1;
    prm.max_halvings = o->max_halvings;
    prm.cap = o->step_cap_cells;
    prm.box = GridDev{box->lo[0], box->lo[1], box->step[0], box->step[1], box->n[0], box->n[1]};
    if (smem_hits < 0) smem_hits = 0;
    if (smem_hits > 12288) smem_hits = 12288;
#define RETINA_LS_CASE(M, PP)                                                                                 \
    return launch_ls_t<M, PP>(hits, n_hits, off, n_events, n_seeds, seeds, prm, smem_hits, theta_out, R_out, status, n_evals, st)
    if (model == RETINA_VELO_SLOPES) {
        if (seeds_per_warp >= 4) RETINA_LS_CASE(RETINA_VELO_SLOPES, 4);
        if (seeds_per_warp == 2) RETINA_LS_CASE(RETINA_VELO_SLOPES, 2);
        RETINA_LS_CASE(RETINA_VELO_SLOPES, 1);
    } else {
        if (seeds_per_warp >= 4) RETINA_LS_CASE(RETINA_TOY2D, 4);
        if (seeds_per_warp == 2) RETINA_LS_CASE(RETINA_TOY2D, 2);
        RETINA_LS_CASE(RETINA_TOY2D, 1);
    }
#undef RETINA_LS_CASE
}

cudaError_t launch_response(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                            const float *theta,
                            int n_points, float sigma, int want_derivs, float *out, cudaStream_t st) {
    const double s = sigma;
    const float kk = (float)(kLog2e / (s * s));
    const float k = (float)(1.0 / (s * s));
    dim3 grid((n_points + 7) / 8, n_events);
    if (model == RETINA_VELO_SLOPES)
        response_kernel<RETINA_VELO_SLOPES><<<grid, 256, 0, st>>>(hits, n_hits, off, n_points, theta, kk, k, want_derivs, out);
    else
        response_kernel<RETINA_TOY2D><<<grid, 256, 0, st>>>(hits, n_hits, off, n_points, theta, kk, k, want_derivs, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace retina
