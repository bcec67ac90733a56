// Multistart local search (Algorithm 1) with the truncated Newton update and
// annealed bandwidth of Section 3 - one launch, one CTA per (event, block of
// seeds) - plus point-wise R / grad R / Hess R.  The per-seed arithmetic is in
// search_device.cuh.
#include "search_device.cuh"

namespace retina {

// One warp owns P consecutive seeds; WARPS warps per CTA share the hits of
// the CTA's event (blockIdx.y), staged once.
template <int MODEL, int P, int WARPS, int UPD>
__global__ void __launch_bounds__(WARPS * 32)
local_search_kernel(const float4 *__restrict__ hits, int64_t n_hits, const int64_t *__restrict__ off,
                    const float4 *__restrict__ boxes, int n_seeds, const float *__restrict__ seeds, LsParams prm,
                    int smem_hits, float *__restrict__ theta_out, float *__restrict__ R_out,
                    uint8_t *__restrict__ status, uint8_t *__restrict__ n_evals, unsigned long long *__restrict__ work) {
    extern __shared__ float4 sh[];
    const int e = blockIdx.y;
    int64_t hb, he;
    event_range(off, n_hits, e, hb, he);
    const int H = (int)(he - hb);
    const float4 *gh = hits + hb;
    const int n_staged = H < smem_hits ? H : smem_hits;
    for (int k = threadIdx.x; k < n_staged; k += blockDim.x) sh[k] = __ldg(gh + k);
    float4 *sbox = staged_box_bounds(sh, smem_hits);
    const int box_cap = default_box_cap(smem_hits);
    float *sz2 = staged_box_z2(sh, smem_hits, box_cap);
    float4 *ssb = staged_super_bounds(sh, smem_hits, box_cap);
    float *ssz2 = staged_super_z2(sh, smem_hits, box_cap);
    const float4 *gbox = boxes ? boxes + 2 * (hb / 32 + e) : nullptr;
    const int n_sbox = gbox ? (((H + 31) >> 5) < box_cap ? ((H + 31) >> 5) : box_cap) : 0;
    stage_boxes<MODEL>(gbox, n_sbox, sbox, sz2, ssb, ssz2, threadIdx.x, blockDim.x);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s_first = (blockIdx.x * WARPS + warp) * P;
    if (s_first >= n_seeds) return;
    const int n_live = n_seeds - s_first < P ? n_seeds - s_first : P;
    const int64_t o = (int64_t)e * n_seeds + s_first;
    search_group<MODEL, P, UPD>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, kept_list(sh, smem_hits, box_cap, warp), seeds + 2 * o,
                           n_live, prm, theta_out + 2 * o, R_out + o,
                           status + o, n_evals ? n_evals + o : nullptr, work);
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

LsParams make_ls_params(const retina_ls_opts *o, const retina_grid *box) {
    LsParams prm;
    prm.q = o->q;
    for (int j = 0; j < RETINA_MAX_Q; ++j) {
        const double s = j < o->q ? (double)o->sigma[j] : 1.0;
        prm.kk[j] = (float)(kLog2e / (s * s));
        prm.k[j] = (float)(1.0 / (s * s));
        prm.cull[j] = (float)((double)CULL_EXPONENT / (double)prm.kk[j]);
    }
    prm.c1 = o->c1;
    prm.max_halvings = o->max_halvings;
    prm.cap = o->step_cap_cells;
    prm.box = GridDev{box->lo[0], box->lo[1], box->step[0], box->step[1], box->n[0], box->n[1]};
    prm.pair_trials = 0;
    return prm;
}

template <int MODEL, int P, int WARPS, int UPD>
static cudaError_t launch_ls_t(const float4 *hits, int64_t n_hits, const int64_t *off, const float4 *boxes,
                               int n_events, int n_seeds, const float *seeds, const LsParams &prm, int smem_hits,
                               float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals, cudaStream_t st) {
    auto kern = local_search_kernel<MODEL, P, WARPS, UPD>;
    const size_t smem = search_smem_bytes(smem_hits, boxes != nullptr, WARPS, default_box_cap(smem_hits));
    cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (aerr != cudaSuccess) return aerr;
    const int per_block = WARPS * P;
    dim3 grid((n_seeds + per_block - 1) / per_block, n_events);
    // latency-bound (at most two warps per warp slot of the GPU): pair the trials
    LsParams p2 = prm;
    p2.pair_trials = (int64_t)grid.x * grid.y * WARPS <= 2LL * sm_count() * 64 ? 1 : 0;
    kern<<<grid, WARPS * 32, smem, st>>>(hits, n_hits, off, boxes, n_seeds, seeds, p2, smem_hits, theta_out, R_out,
                                         status, n_evals, work_counters());
    count_launches(1);
    return cudaGetLastError();
}

template <int MODEL, int P, int UPD = RETINA_UPDATE_TRUNCATED_NEWTON>
static cudaError_t launch_ls_w(int warps, const float4 *hits, int64_t n_hits, const int64_t *off, const float4 *boxes,
                               int n_events, int n_seeds, const float *seeds, const LsParams &prm, int smem_hits,
                               float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals, cudaStream_t st) {
    if (warps >= 16)
        return launch_ls_t<MODEL, P, 16, UPD>(hits, n_hits, off, boxes, n_events, n_seeds, seeds, prm, smem_hits,
                                              theta_out, R_out, status, n_evals, st);
    if (warps >= 8)
        return launch_ls_t<MODEL, P, 8, UPD>(hits, n_hits, off, boxes, n_events, n_seeds, seeds, prm, smem_hits,
                                             theta_out, R_out, status, n_evals, st);
    return launch_ls_t<MODEL, P, 4, UPD>(hits, n_hits, off, boxes, n_events, n_seeds, seeds, prm, smem_hits,
                                         theta_out, R_out, status, n_evals, st);
}

cudaError_t launch_local_search(const float4 *hits, int64_t n_hits, const int64_t *off, const float4 *boxes,
                                int n_events, int model, const float *seeds, int n_seeds, const retina_ls_opts *o, const retina_grid *box,
                                float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals, int seeds_per_warp,
                                int warps, int smem_hits, cudaStream_t st) {
    LsParams prm = make_ls_params(o, box);
    if (smem_hits < 0) smem_hits = 0;
    if (smem_hits > 12288) smem_hits = 12288;
    // the comparison updates run one seed per warp (the same results as any
    // other grouping), which keeps their instantiations few
#define RETINA_LS_ALT(M, U)                                                                                           \
    return launch_ls_w<M, 1, U>(warps, hits, n_hits, off, boxes, n_events, n_seeds, seeds, prm, smem_hits, theta_out, \
                                R_out, status, n_evals, st)
    if (o->update == RETINA_UPDATE_STEEPEST_ASCENT) {
        if (model == RETINA_VELO_SLOPES) RETINA_LS_ALT(RETINA_VELO_SLOPES, RETINA_UPDATE_STEEPEST_ASCENT);
        RETINA_LS_ALT(RETINA_TOY2D, RETINA_UPDATE_STEEPEST_ASCENT);
    }
    if (o->update == RETINA_UPDATE_MODIFIED_NEWTON) {
        if (model == RETINA_VELO_SLOPES) RETINA_LS_ALT(RETINA_VELO_SLOPES, RETINA_UPDATE_MODIFIED_NEWTON);
        RETINA_LS_ALT(RETINA_TOY2D, RETINA_UPDATE_MODIFIED_NEWTON);
    }
#undef RETINA_LS_ALT
#define RETINA_LS_CASE(M, PP)                                                                                     \
    return launch_ls_w<M, PP>(warps, hits, n_hits, off, boxes, n_events, n_seeds, seeds, prm, smem_hits, theta_out, \
                              R_out, status, n_evals, st)
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
