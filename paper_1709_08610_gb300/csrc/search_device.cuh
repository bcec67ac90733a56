// Device side of the multistart search (Algorithm 1 with the truncated Newton
// update of Section 3), shared by the per-launch kernel (local_search.cu) and
// the persistent batched kernel (batched_search.cu) so both run identical
// arithmetic.
//
// Layout: one warp owns P seeds of one event; its 32 lanes stride over the
// event's hits (staged in shared memory, float4 per hit; hits beyond the
// staged capacity are read through L1/L2), each lane accumulating the sums of
// Eq. 1 and its derivatives for all P seeds, then a xor-butterfly reduction
// leaves bitwise-identical totals in every lane.  Every decision (CG branch,
// step cap, Armijo test) is therefore warp-uniform: no lane ever diverges
// from its warp, and seeds that finished their line search idle under a
// uniform predicate.
//
// Sums per pair, with e = exp(-|r|^2 / sigma^2), k = 1 / sigma^2:
//   slope model (J = z I):     S = [e, e z rx, e z ry, e z^2 rx^2, e z^2 rx ry, e z^2 ry^2, e z^2]
//     grad = 2k (S1, S2);  H = 4k^2 [S3 S4; S4 S5] - 2k S6 I
//   2D toy (J = [x, 1]):       S = [e, e r x, e r, e r^2 x^2, e r^2 x, e r^2, e x^2, e x]
//     grad = 2k (S1, S2);  H = 4k^2 [S3 S4; S4 S5] - 2k [S6 S7; S7 S0]
#pragma once

#include "internal.cuh"

namespace retina {

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

LsParams make_ls_params(const retina_ls_opts *o, const retina_grid *box);

// Lane-strided pass over an event's hits: the staged prefix from shared
// memory (two hits per iteration for independent work), then the rest, if
// any, straight from global memory through L1.
template <typename F>
__device__ __forceinline__ void for_each_hit(const float4 *__restrict__ sh, const float4 *__restrict__ gh,
                                             int n_staged, int H, int lane, F &&f) {
    int k = lane;
    for (; k + 32 < n_staged; k += 64) {
        const float4 a = sh[k], b = sh[k + 32];
        f(a);
        f(b);
    }
    for (; k < n_staged; k += 32) f(sh[k]);
    for (; k < H; k += 32) f(__ldg(gh + k));
}

// Algorithm 1 for the P seeds of one warp: q truncated-Newton updates
// (gradient/Hessian pass, Newton-CG direction, step cap, Armijo backtracking
// at bandwidth sigma_j), then R(theta_q; sigma_q), status and the number of
// R-only passes.  seeds / outputs point at the group's first seed; only the
// first n_live (<= P) seeds exist.  Warp-uniform control flow throughout.
template <int MODEL, int P>
__device__ __forceinline__ void search_group(const float4 *__restrict__ sh, const float4 *__restrict__ gh,
                                             int n_staged, int H, int lane, const float *__restrict__ seeds,
                                             int n_live, const LsParams &prm, float *__restrict__ theta_out,
                                             float *__restrict__ R_out, uint8_t *__restrict__ status,
                                             uint8_t *__restrict__ n_evals) {
    constexpr int NS = Model<MODEL>::NS;
    float th0[P], th1[P], Rfin[P];
    int evals[P];
    bool live[P], failed[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        live[p] = p < n_live;
        const int o = (live[p] ? p : 0) * 2;
        th0[p] = seeds[o];
        th1[p] = seeds[o + 1];
        failed[p] = false;
        evals[p] = 0;
        Rfin[p] = 0.f;
    }

    for (int j = 0; j < prm.q; ++j) {
        const float kk = prm.kk[j], k = prm.k[j];
        // (R, g, H) at the current points
        float S[P][NS];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < NS; ++i) S[p][i] = 0.f;
        for_each_hit(sh, gh, n_staged, H, lane, [&](const float4 h) {
#pragma unroll
            for (int p = 0; p < P; ++p) pair_rgh<MODEL>(h, th0[p], th1[p], kk, S[p]);
        });
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
            Rfin[p] = R[p];  // R at the point if no step is accepted
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
            for_each_hit(sh, gh, n_staged, H, lane, [&](const float4 h) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (pending[p]) Rt[p] += pair_r<MODEL>(h, tr0[p], tr1[p], kk);
            });
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (!pending[p]) continue;
                ++evals[p];
                const float rt = warp_sum(Rt[p]);
                if (rt >= R[p] + prm.c1 * t[p] * slope[p]) {
                    th0[p] = tr0[p];
                    th1[p] = tr1[p];
                    Rfin[p] = rt;  // R at the accepted point, this update's bandwidth
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

    // After the last update Rfin holds R(theta_q; sigma_q): the accepted
    // trial's response, or the response at the unmoved point - the same sum,
    // in the same order, that a separate evaluation would produce.
    const float hi0 = prm.box.lo0 + (float)prm.box.n0 * prm.box.step0;
    const float hi1 = prm.box.lo1 + (float)prm.box.n1 * prm.box.step1;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!live[p] || lane != 0) continue;
        uint8_t st;
        if (!(isfinite(th0[p]) && isfinite(th1[p]) && isfinite(Rfin[p])))
            st = 3;
        else if (!(th0[p] >= prm.box.lo0 && th0[p] < hi0 && th1[p] >= prm.box.lo1 && th1[p] < hi1))
            st = 2;
        else
            st = failed[p] ? 1 : 0;
        theta_out[2 * p] = th0[p];
        theta_out[2 * p + 1] = th1[p];
        R_out[p] = Rfin[p];
        status[p] = st;
        if (n_evals) n_evals[p] = (uint8_t)(evals[p] < 255 ? evals[p] : 255);
    }
}

}  // namespace retina
