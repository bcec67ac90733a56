// C ABI entry points (declared in include/retina.h): host-side validation,
// workspace layout and launch.  No entry point allocates device memory.
#include <math.h>

#include <atomic>

#include "internal.cuh"

namespace retina {

static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

static std::atomic<int> g_opt_seeds_per_warp{1};
static std::atomic<int> g_opt_smem_hits{4096};
static std::atomic<int> g_opt_grid_splits{0};
static std::atomic<int> g_opt_ls_warps{8};
static std::atomic<int> g_opt_batch_spw{1};
static std::atomic<int> g_opt_batch_warps{16};
static std::atomic<int> g_opt_batch_smem_hits{8192};
static std::atomic<int> g_opt_batch_ctas{0};
static std::atomic<int> g_opt_seednet_tc{1};
static std::atomic<int> g_opt_grid_tc{1};

int option_value(int option) {
    int32_t v = 0;
    return retina_get_option(option, &v) == RETINA_OK ? v : 0;
}

static bool finite_pos(float v) { return isfinite(v) && v > 0.f; }

static bool valid_grid(const retina_grid *g) {
    if (!g) return false;
    for (int a = 0; a < 2; ++a) {
        if (!isfinite(g->lo[a]) || !finite_pos(g->step[a]) || g->n[a] <= 0) return false;
        if (!isfinite(g->lo[a] + (float)g->n[a] * g->step[a])) return false;
    }
    return (int64_t)g->n[0] * (int64_t)g->n[1] <= (int64_t)INT32_MAX;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct GridWs {
    size_t R_off, R_bytes, part_off, part_bytes, max_off, max_bytes, total;
};

static GridWs grid_ws_layout(const GridPlan &p, int n_events, const retina_grid *g, bool store_R) {
    GridWs w;
    const size_t cells = (size_t)g->n[0] * (size_t)g->n[1];
    w.R_off = 0;
    w.R_bytes = store_R ? 0 : round_up(cells * (size_t)n_events * sizeof(float), 256);
    w.part_off = w.R_off + w.R_bytes;
    w.part_bytes = round_up(grid_partials_bytes(p, n_events, g), 256);
    w.max_off = w.part_off + w.part_bytes;
    w.max_bytes = round_up(maxima_ws_bytes(n_events, g), 256);
    w.total = w.max_off + w.max_bytes;
    return w;
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? RETINA_OK : RETINA_ECUDA; }

}  // namespace retina

using namespace retina;

extern "C" {

const char *retina_strerror(int code) {
    switch (code) {
        case RETINA_OK: return "ok";
        case RETINA_EINVAL: return "invalid argument (nothing launched)";
        case RETINA_ECUDA: return "CUDA launch or runtime error";
        case RETINA_ENOSPACE: return "workspace too small or size limit exceeded";
        default: return "unknown retina status";
    }
}

int retina_abi_version(void) { return 2; }

int retina_set_option(int32_t option, int32_t value) {
    switch (option) {
        case RETINA_OPT_LS_SEEDS_PER_WARP:
            if (value != 1 && value != 2 && value != 4) return RETINA_EINVAL;
            g_opt_seeds_per_warp = value;
            return RETINA_OK;
        case RETINA_OPT_LS_SMEM_HITS:
            if (value < 0 || value > 12288) return RETINA_EINVAL;
            g_opt_smem_hits = value;
            return RETINA_OK;
        case RETINA_OPT_GRID_SPLITS:
            if (value < 0 || value > 64) return RETINA_EINVAL;
            g_opt_grid_splits = value;
            return RETINA_OK;
        case RETINA_OPT_LS_WARPS:
            if (value != 4 && value != 8 && value != 16) return RETINA_EINVAL;
            g_opt_ls_warps = value;
            return RETINA_OK;
        case RETINA_OPT_BATCH_SEEDS_PER_WARP:
            if (value != 1 && value != 2 && value != 4) return RETINA_EINVAL;
            g_opt_batch_spw = value;
            return RETINA_OK;
        case RETINA_OPT_BATCH_WARPS:
            if (value != 8 && value != 16 && value != 32) return RETINA_EINVAL;
            g_opt_batch_warps = value;
            return RETINA_OK;
        case RETINA_OPT_BATCH_SMEM_HITS:
            if (value < 0 || value > 12288) return RETINA_EINVAL;
            g_opt_batch_smem_hits = value;
            return RETINA_OK;
        case RETINA_OPT_BATCH_CTAS:
            if (value < 0 || value > (1 << 20)) return RETINA_EINVAL;
            g_opt_batch_ctas = value;
            return RETINA_OK;
        case RETINA_OPT_SEEDNET_TC:
            if (value != 0 && value != 1) return RETINA_EINVAL;
            g_opt_seednet_tc = value;
            return RETINA_OK;
        case RETINA_OPT_GRID_TC:
            if (value != 0 && value != 1) return RETINA_EINVAL;
            g_opt_grid_tc = value;
            return RETINA_OK;
        default: return RETINA_EINVAL;
    }
}

int retina_get_option(int32_t option, int32_t *value) {
    if (!value) return RETINA_EINVAL;
    switch (option) {
        case RETINA_OPT_LS_SEEDS_PER_WARP: *value = g_opt_seeds_per_warp; return RETINA_OK;
        case RETINA_OPT_LS_SMEM_HITS: *value = g_opt_smem_hits; return RETINA_OK;
        case RETINA_OPT_GRID_SPLITS: *value = g_opt_grid_splits; return RETINA_OK;
        case RETINA_OPT_LS_WARPS: *value = g_opt_ls_warps; return RETINA_OK;
        case RETINA_OPT_BATCH_SEEDS_PER_WARP: *value = g_opt_batch_spw; return RETINA_OK;
        case RETINA_OPT_BATCH_WARPS: *value = g_opt_batch_warps; return RETINA_OK;
        case RETINA_OPT_BATCH_SMEM_HITS: *value = g_opt_batch_smem_hits; return RETINA_OK;
        case RETINA_OPT_BATCH_CTAS: *value = g_opt_batch_ctas; return RETINA_OK;
        case RETINA_OPT_SEEDNET_TC: *value = g_opt_seednet_tc; return RETINA_OK;
        case RETINA_OPT_GRID_TC: *value = g_opt_grid_tc; return RETINA_OK;
        default: return RETINA_EINVAL;
    }
}

int retina_grid_scan_workspace_size(int32_t n_events, int32_t model, const retina_grid *g, int32_t flags,
                                    int32_t store_R, size_t *bytes) {
    if (!bytes || n_events < 0 || !valid_grid(g)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (flags < RETINA_GRID_AUTO || flags > RETINA_GRID_TENSOR) return RETINA_EINVAL;
    if (flags >= RETINA_GRID_SEPARABLE && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    const GridPlan p = plan_grid(n_events, model, g, flags, g_opt_grid_splits);
    *bytes = grid_ws_layout(p, n_events, g, store_R != 0).total;
    return RETINA_OK;
}

int retina_grid_scan(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events, int32_t model,
                     const retina_grid *g, float sigma, float R0, int32_t flags, float *R_out, int32_t *max_idx,
                     float *max_theta, float *max_R, int32_t *n_max, int32_t K, void *ws, size_t ws_bytes,
                     void *stream) {
    if (n_events < 0 || n_hits < 0 || !valid_grid(g) || !finite_pos(sigma) || isnan(R0) || K < 1)
        return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (flags < RETINA_GRID_AUTO || flags > RETINA_GRID_TENSOR) return RETINA_EINVAL;
    if (flags >= RETINA_GRID_SEPARABLE && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !max_idx || !max_theta || !max_R || !n_max) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    if (R_out && !aligned16(R_out)) return RETINA_EINVAL;
    const GridPlan p = plan_grid(n_events, model, g, flags, g_opt_grid_splits);
    const GridWs w = grid_ws_layout(p, n_events, g, R_out != nullptr);
    if (ws_bytes < w.total) return RETINA_ENOSPACE;
    if (w.total > 0 && (!ws || ((uintptr_t)ws & 255u))) return RETINA_EINVAL;
    char *base = (char *)ws;
    float *R = R_out ? R_out : (float *)(base + w.R_off);
    float *partials = (float *)(base + w.part_off);
    int32_t *mws = (int32_t *)(base + w.max_off);
    cudaStream_t st = (cudaStream_t)stream;
    if (boxes && !aligned16(boxes)) return RETINA_EINVAL;
    cudaError_t err = launch_grid_response(p, (const float4 *)hits, n_hits, event_offsets, (const float4 *)boxes,
                                           n_events, model, g, sigma, R, partials, st);
    if (err != cudaSuccess) return RETINA_ECUDA;
    return cuda_status(launch_grid_maxima(R, n_events, g, R0, max_idx, max_theta, max_R, n_max, K, mws, st));
}

int retina_grid_response_workspace_size(int32_t n_events, int32_t model, const retina_grid *g, int32_t flags,
                                        size_t *bytes) {
    if (!bytes || n_events < 0 || !valid_grid(g)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (flags < RETINA_GRID_AUTO || flags > RETINA_GRID_TENSOR) return RETINA_EINVAL;
    if (flags >= RETINA_GRID_SEPARABLE && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    const GridPlan p = plan_grid(n_events, model, g, flags, g_opt_grid_splits);
    *bytes = round_up(grid_partials_bytes(p, n_events, g), 256);
    return RETINA_OK;
}

int retina_grid_response(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events,
                         int32_t model, const retina_grid *g, float sigma, int32_t flags, float *R_out, void *ws,
                         size_t ws_bytes, void *stream) {
    if (n_events < 0 || n_hits < 0 || !valid_grid(g) || !finite_pos(sigma)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (flags < RETINA_GRID_AUTO || flags > RETINA_GRID_TENSOR) return RETINA_EINVAL;
    if (flags >= RETINA_GRID_SEPARABLE && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !R_out || !aligned16(R_out)) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    const GridPlan p = plan_grid(n_events, model, g, flags, g_opt_grid_splits);
    const size_t need = round_up(grid_partials_bytes(p, n_events, g), 256);
    if (ws_bytes < need) return RETINA_ENOSPACE;
    if (need > 0 && (!ws || ((uintptr_t)ws & 255u))) return RETINA_EINVAL;
    if (boxes && !aligned16(boxes)) return RETINA_EINVAL;
    return cuda_status(launch_grid_response(p, (const float4 *)hits, n_hits, event_offsets, (const float4 *)boxes,
                                            n_events, model, g, sigma, R_out, (float *)ws, (cudaStream_t)stream));
}

int64_t retina_prepare_hits_box_count(int64_t n_hits, int32_t n_events) {
    if (n_hits < 0 || n_events < 0) return -1;
    return prepared_box_count(n_hits, n_events);
}

int retina_prepare_hits(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                        int32_t model, float *sorted_out, float *boxes_out, void *stream) {
    if (n_events < 0 || n_hits < 0) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !boxes_out || !aligned16(boxes_out)) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !sorted_out || !aligned16(hits) || !aligned16(sorted_out))) return RETINA_EINVAL;
    if (n_hits > 0 && hits == sorted_out) return RETINA_EINVAL;  // not in place
    return cuda_status(launch_prepare_hits((const float4 *)hits, n_hits, event_offsets, n_events, model,
                                           (float4 *)sorted_out, (float4 *)boxes_out, (cudaStream_t)stream));
}

uint64_t retina_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int retina_grid_maxima_workspace_size(int32_t n_events, const retina_grid *g, size_t *bytes) {
    if (!bytes || n_events < 0 || !valid_grid(g)) return RETINA_EINVAL;
    *bytes = round_up(maxima_ws_bytes(n_events, g), 256);
    return RETINA_OK;
}

int retina_grid_maxima(const float *R, int32_t n_events, const retina_grid *g, float R0, int32_t *max_idx,
                       float *max_theta, float *max_R, int32_t *n_max, int32_t K, void *ws, size_t ws_bytes,
                       void *stream) {
    if (n_events < 0 || !valid_grid(g) || isnan(R0) || K < 1) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!R || !max_idx || !max_theta || !max_R || !n_max) return RETINA_EINVAL;
    const size_t need = round_up(maxima_ws_bytes(n_events, g), 256);
    if (ws_bytes < need) return RETINA_ENOSPACE;
    if (!ws || ((uintptr_t)ws & 255u)) return RETINA_EINVAL;
    return cuda_status(launch_grid_maxima(R, n_events, g, R0, max_idx, max_theta, max_R, n_max, K, (int32_t *)ws,
                                          (cudaStream_t)stream));
}

int retina_response(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events, int32_t model,
                    const float *theta, int32_t n_points, float sigma, int32_t want_derivs, float *out, void *stream) {
    if (n_events < 0 || n_points < 0 || n_hits < 0 || !finite_pos(sigma)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events == 0 || n_points == 0) return RETINA_OK;
    if (!event_offsets || !theta || !out) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    if ((int64_t)n_events * 65535 < 0 || n_events > 65535) return RETINA_EINVAL;
    return cuda_status(launch_response((const float4 *)hits, n_hits, event_offsets, n_events, model, theta, n_points,
                                       sigma, want_derivs != 0, out, (cudaStream_t)stream));
}

static bool valid_ls_opts(const retina_ls_opts *opts) {
    if (!opts || opts->q < 1 || opts->q > RETINA_MAX_Q) return false;
    for (int j = 0; j < opts->q; ++j)
        if (!finite_pos(opts->sigma[j])) return false;
    if (!(opts->c1 >= 0.f && opts->c1 < 1.f)) return false;
    if (opts->max_halvings < 0 || opts->max_halvings > 30) return false;
    if (opts->update < RETINA_UPDATE_TRUNCATED_NEWTON || opts->update > RETINA_UPDATE_MODIFIED_NEWTON) return false;
    return opts->step_cap_cells > 0.f;
}

int retina_local_search(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events,
                        int32_t model, const float *seeds, int32_t n_seeds, const retina_ls_opts *opts,
                        const retina_grid *box, float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals,
                        void *stream) {
    if (n_events < 0 || n_seeds < 0 || n_hits < 0 || !valid_ls_opts(opts) || !valid_grid(box)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events > 65535) return RETINA_EINVAL;
    if (n_events == 0 || n_seeds == 0) return RETINA_OK;
    if (!event_offsets || !seeds || !theta_out || !R_out || !status) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    if (boxes && !aligned16(boxes)) return RETINA_EINVAL;
    return cuda_status(launch_local_search((const float4 *)hits, n_hits, event_offsets, (const float4 *)boxes,
                                           n_events, model, seeds,
                                           n_seeds, opts, box, theta_out, R_out, status, n_evals, g_opt_seeds_per_warp,
                                           g_opt_ls_warps, g_opt_smem_hits, (cudaStream_t)stream));
}

int retina_refine_maxima_workspace_size(int32_t n_events, size_t *bytes) {
    if (!bytes || n_events < 0) return RETINA_EINVAL;
    *bytes = batched_ws_bytes(n_events);
    return RETINA_OK;
}

int retina_refine_maxima(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes,
                         int32_t n_events, int32_t model, const float *theta_c, const int32_t *n_max, int32_t K,
                         const retina_ls_opts *opts, const retina_grid *box, float *theta_out, float *R_out,
                         uint8_t *status, void *ws, size_t ws_bytes, void *stream) {
    if (n_events < 0 || K < 0 || n_hits < 0 || !valid_ls_opts(opts) || !valid_grid(box)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_events > 65535) return RETINA_EINVAL;
    if (n_events == 0 || K == 0) return RETINA_OK;
    if (!event_offsets || !theta_c || !n_max || !theta_out || !R_out || !status) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    if (boxes && !aligned16(boxes)) return RETINA_EINVAL;
    if (ws_bytes < batched_ws_bytes(n_events)) return RETINA_ENOSPACE;
    if (!ws || ((uintptr_t)ws & 255u)) return RETINA_EINVAL;
    return cuda_status(launch_refine_maxima((const float4 *)hits, n_hits, event_offsets, (const float4 *)boxes,
                                            n_events, model, theta_c, n_max, K, opts, box, theta_out, R_out, status,
                                            (int32_t *)ws, g_opt_batch_spw, g_opt_batch_warps, g_opt_batch_smem_hits,
                                            g_opt_batch_ctas, (cudaStream_t)stream));
}

int retina_local_search4(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                         const float *seeds, int32_t n_seeds, const int32_t *seed_count, const retina_ls4_opts *opts,
                         float *theta_out, float *R_out, uint8_t *status, void *stream) {
    if (n_events < 0 || n_seeds < 0 || n_hits < 0 || !opts) return RETINA_EINVAL;
    if (opts->q < 1 || opts->q > RETINA_MAX_Q) return RETINA_EINVAL;
    for (int j = 0; j < opts->q; ++j)
        if (!finite_pos(opts->sigma[j])) return RETINA_EINVAL;
    if (!(opts->c1 >= 0.f && opts->c1 < 1.f) || opts->max_halvings < 0 || opts->max_halvings > 30) return RETINA_EINVAL;
    for (int a = 0; a < 4; ++a)
        if (!finite_pos(opts->scale[a])) return RETINA_EINVAL;
    if (!(opts->step_cap > 0.f) || !isfinite(opts->zref)) return RETINA_EINVAL;
    if (n_events > 65535) return RETINA_EINVAL;
    if (n_events == 0 || n_seeds == 0) return RETINA_OK;
    if (!event_offsets || !seeds || !theta_out || !R_out || !status) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    return cuda_status(launch_local_search4((const float4 *)hits, n_hits, event_offsets, n_events, seeds, n_seeds,
                                            seed_count, opts, theta_out, R_out, status, g_opt_smem_hits,
                                            (cudaStream_t)stream));
}

int retina_pair_seeds4(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                       const float *layer_z, int32_t n_pairs, float dz_tol, float d_max, float zc_lo, float zc_hi,
                       float zref, float *seeds, int32_t *n_seeds, int32_t K, void *stream) {
    if (n_events < 0 || n_hits < 0 || K < 1 || n_pairs < 1 || n_pairs > RETINA_MAX_LAYER_PAIRS) return RETINA_EINVAL;
    if (!(isfinite(dz_tol) && dz_tol >= 0.f) || !(isfinite(d_max) && d_max >= 0.f) || !isfinite(zc_lo) ||
        !isfinite(zc_hi) || !isfinite(zref) || !layer_z)
        return RETINA_EINVAL;
    for (int p = 0; p < 2 * n_pairs; ++p)
        if (!isfinite(layer_z[p])) return RETINA_EINVAL;
    if ((int64_t)K * 4 > (int64_t)INT32_MAX) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !seeds || !n_seeds) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    return cuda_status(launch_pair_seeds4((const float4 *)hits, n_hits, event_offsets, n_events, layer_z, n_pairs,
                                          dz_tol, d_max, zc_lo, zc_hi, zref, seeds, n_seeds, K, (cudaStream_t)stream));
}

int retina_batched_search_workspace_size(int32_t n_events, size_t *bytes) {
    if (!bytes || n_events < 0) return RETINA_EINVAL;
    *bytes = batched_ws_bytes(n_events);
    return RETINA_OK;
}

int retina_batched_search(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events,
                          int32_t model, const float *seeds, int64_t n_seeds, const int64_t *seed_offsets,
                          const int32_t *order, const retina_ls_opts *opts, const retina_grid *box, float *theta_out,
                          float *R_out, uint8_t *status, uint8_t *n_evals, void *ws, size_t ws_bytes, void *stream) {
    if (n_events < 0 || n_seeds < 0 || n_hits < 0 || !valid_ls_opts(opts) || !valid_grid(box)) return RETINA_EINVAL;
    if (model != RETINA_TOY2D && model != RETINA_VELO_SLOPES) return RETINA_EINVAL;
    if (n_seeds > (int64_t)INT32_MAX) return RETINA_EINVAL;
    if (n_events == 0 || n_seeds == 0) return RETINA_OK;
    if (!event_offsets || !seed_offsets || !seeds || !theta_out || !R_out || !status) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    if (ws_bytes < batched_ws_bytes(n_events)) return RETINA_ENOSPACE;
    if (!ws || ((uintptr_t)ws & 255u)) return RETINA_EINVAL;
    if (boxes && !aligned16(boxes)) return RETINA_EINVAL;
    return cuda_status(launch_batched_search((const float4 *)hits, n_hits, event_offsets, (const float4 *)boxes,
                                             n_events, model, seeds,
                                             n_seeds, seed_offsets, order, opts, box, theta_out, R_out, status,
                                             n_evals, (int32_t *)ws, g_opt_batch_spw, g_opt_batch_warps,
                                             g_opt_batch_smem_hits, g_opt_batch_ctas, (cudaStream_t)stream));
}

int retina_sort_seeds(const float *seeds, int64_t n_seeds, const int64_t *seed_offsets, int32_t n_events,
                      const retina_grid *box, float *sorted_out, int32_t *perm_out, void *stream) {
    if (n_events < 0 || n_seeds < 0 || !valid_grid(box)) return RETINA_EINVAL;
    if (n_events == 0 || n_seeds == 0) return RETINA_OK;
    if (!seeds || !seed_offsets || !sorted_out || seeds == sorted_out) return RETINA_EINVAL;
    if (((uintptr_t)seeds & 7u) || ((uintptr_t)sorted_out & 7u)) return RETINA_EINVAL;
    return cuda_status(launch_sort_seeds(seeds, n_seeds, seed_offsets, n_events, box, sorted_out, perm_out,
                                         (cudaStream_t)stream));
}

int retina_extract_tracks(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                          int32_t n_events, int32_t n_points, const retina_grid *box, float R0, float merge_cells,
                          float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int32_t K,
                          void *stream) {
    if (n_events < 0 || n_points < 0 || !valid_grid(box) || isnan(R0) || !finite_pos(merge_cells) || K < 1)
        return RETINA_EINVAL;
    for (int a = 0; a < 2; ++a)
        if ((double)box->n[a] / (double)merge_cells > 32768.0) return RETINA_EINVAL;
    if (n_points > RETINA_MAX_EXTRACT_POINTS) return RETINA_ENOSPACE;
    if (n_events == 0) return RETINA_OK;
    if (!n_tracks) return RETINA_EINVAL;
    if (n_points > 0 && (!theta || !R)) return RETINA_EINVAL;
    if (!tracks || !track_R) return RETINA_EINVAL;
    return cuda_status(launch_extract_tracks(theta, R, status, n_valid, n_events, n_points, box, R0, merge_cells,
                                             tracks, track_R, track_src, n_tracks, K, (cudaStream_t)stream));
}

int retina_extract_tracks_workspace_size(int32_t n_events, int32_t n_points, size_t *bytes) {
    if (!bytes || n_events < 0 || n_points < 0 || n_points > RETINA_MAX_EXTRACT_POINTS_WS) return RETINA_EINVAL;
    *bytes = n_points > RETINA_MAX_EXTRACT_POINTS ? (size_t)n_events * extract_ws_stride(n_points, 2) : 0;
    return RETINA_OK;
}

int retina_extract_tracks_ws(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                             int32_t n_events, int32_t n_points, const retina_grid *box, float R0, float merge_cells,
                             float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int32_t K,
                             void *ws, size_t ws_bytes, void *stream) {
    if (n_points <= RETINA_MAX_EXTRACT_POINTS)
        return retina_extract_tracks(theta, R, status, n_valid, n_events, n_points, box, R0, merge_cells, tracks,
                                     track_R, track_src, n_tracks, K, stream);
    if (n_events < 0 || !valid_grid(box) || isnan(R0) || !finite_pos(merge_cells) || K < 1) return RETINA_EINVAL;
    for (int a = 0; a < 2; ++a)
        if ((double)box->n[a] / (double)merge_cells > 32768.0) return RETINA_EINVAL;
    if (n_points > RETINA_MAX_EXTRACT_POINTS_WS || n_events > 65535) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (ws_bytes < (size_t)n_events * extract_ws_stride(n_points, 2)) return RETINA_ENOSPACE;
    if (!ws || ((uintptr_t)ws & 255u) || !n_tracks || !theta || !R || !tracks || !track_R) return RETINA_EINVAL;
    return cuda_status(launch_extract_tracks(theta, R, status, n_valid, n_events, n_points, box, R0, merge_cells,
                                             tracks, track_R, track_src, n_tracks, K, (cudaStream_t)stream, ws));
}

int retina_extract_tracks4(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                           int32_t n_events, int32_t n_points, const retina_grid *slope_box, const float *unit, float R0,
                           float merge_units, float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks,
                           int32_t K, void *stream) {
    if (n_events < 0 || n_points < 0 || K < 1 || !slope_box || !unit || isnan(R0)) return RETINA_EINVAL;
    if (!(isfinite(merge_units) && merge_units > 0.f)) return RETINA_EINVAL;
    for (int a = 0; a < 4; ++a)
        if (!(isfinite(unit[a]) && unit[a] > 0.f) || !isfinite(merge_units * unit[a])) return RETINA_EINVAL;
    for (int a = 0; a < 2; ++a) {
        if (!isfinite(slope_box->lo[a]) || !(isfinite(slope_box->step[a]) && slope_box->step[a] > 0.f) ||
            slope_box->n[a] <= 0)
            return RETINA_EINVAL;
        // buckets of the slope coordinates are indexed in 21 bits
        if ((double)slope_box->n[a] * slope_box->step[a] / ((double)merge_units * unit[2 + a]) > 1048576.0)
            return RETINA_EINVAL;
    }
    if (n_events == 0) return RETINA_OK;
    if (n_events > 65535) return RETINA_EINVAL;
    if (n_points > RETINA_MAX_EXTRACT_POINTS4) return RETINA_ENOSPACE;
    if (!theta || !R || !tracks || !track_R || !n_tracks) return RETINA_EINVAL;
    return cuda_status(launch_extract_tracks4(theta, R, status, n_valid, n_events, n_points, slope_box, unit, R0,
                                              merge_units, tracks, track_R, track_src, n_tracks, K,
                                              (cudaStream_t)stream));
}

int retina_slope_histogram(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                           float lo, float hi, float zmin, uint16_t *features, int32_t *counts, void *stream) {
    if (n_events < 0 || n_hits < 0 || !isfinite(lo) || !isfinite(hi) || !(lo < hi) || !(zmin >= 0.f))
        return RETINA_EINVAL;
    if (!isfinite(64.f / (hi - lo))) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !features) return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || !aligned16(hits))) return RETINA_EINVAL;
    return cuda_status(launch_slope_hist((const float4 *)hits, n_hits, event_offsets, n_events, lo, hi, zmin,
                                         features, counts, (cudaStream_t)stream));
}

int retina_seednet_forward(const uint16_t *features, int32_t n_events, const float *params, float *logits,
                           uint16_t *h1, uint16_t *h2, void *stream) {
    if (n_events < 0 || n_events > 65535) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!features || !params || !logits || !h1) return RETINA_EINVAL;
    return cuda_status(launch_seednet_forward(features, n_events, params, logits, h1, h2, (cudaStream_t)stream));
}

static bool valid_adam(int32_t step, float lr, float b1, float b2, float eps) {
    return step >= 1 && isfinite(lr) && b1 > 0.f && b1 < 1.f && b2 > 0.f && b2 < 1.f && eps >= 0.f && isfinite(eps);
}

int retina_seednet_train_workspace_size(int32_t n_events, size_t *bytes) {
    if (!bytes || n_events < 0 || n_events > 65535) return RETINA_EINVAL;
    *bytes = seednet_train_ws_bytes(n_events);
    return RETINA_OK;
}

int retina_seednet_train_step(const uint16_t *features, const uint8_t *labels, int32_t n_events, float *params,
                              float *adam_m, float *adam_v, int32_t step, float lr, float beta1, float beta2,
                              float eps, float *loss, float *grad, void *ws, size_t ws_bytes, void *stream) {
    if (n_events < 1 || n_events > 65535 || !valid_adam(step, lr, beta1, beta2, eps)) return RETINA_EINVAL;
    if (!features || !labels || !params || !adam_m || !adam_v) return RETINA_EINVAL;
    if (ws_bytes < seednet_train_ws_bytes(n_events)) return RETINA_ENOSPACE;
    if (!ws || ((uintptr_t)ws & 255u)) return RETINA_EINVAL;
    return cuda_status(launch_seednet_train_step(features, labels, n_events, params, adam_m, adam_v, step, lr, beta1,
                                                 beta2, eps, loss, grad, ws, (cudaStream_t)stream));
}

int retina_seednet_adam(float *params, float *adam_m, float *adam_v, const float *grad, int32_t step, float lr,
                        float beta1, float beta2, float eps, void *stream) {
    if (!valid_adam(step, lr, beta1, beta2, eps)) return RETINA_EINVAL;
    if (!params || !adam_m || !adam_v || !grad) return RETINA_EINVAL;
    return cuda_status(launch_seednet_adam(params, adam_m, adam_v, grad, step, lr, beta1, beta2, eps,
                                           (cudaStream_t)stream));
}

int retina_topk_seeds(const float *logits, int32_t n_events, int32_t K, float lo, float hi, float zmin,
                      int32_t min_sub_hits, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                      float *seeds, int32_t *cell_idx, void *stream) {
    if (n_events < 0 || K < 1 || K > RETINA_SEEDNET_BINS * RETINA_SEEDNET_BINS) return RETINA_EINVAL;
    if (!isfinite(lo) || !isfinite(hi) || !(lo < hi) || !isfinite(256.f / (hi - lo))) return RETINA_EINVAL;
    if (!(zmin >= 0.f) || min_sub_hits < 1 || n_hits < 0) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!logits || !seeds || !aligned16(logits)) return RETINA_EINVAL;
    if (hits && (!event_offsets || !aligned16(hits))) return RETINA_EINVAL;
    return cuda_status(launch_propose_seeds(logits, n_events, K, lo, hi, zmin, min_sub_hits, (const float4 *)hits,
                                            hits ? n_hits : 0, event_offsets, seeds, cell_idx,
                                            (cudaStream_t)stream));
}

}  // extern "C"
