// Native executor of the whole path for a batch of events (retina_pipeline_*):
// hit ordering, then the grid method and Algorithm 1 on two concurrent
// streams, joined into the caller's stream.  Creation validates the
// configuration and allocates every buffer a run needs; a run only enqueues
// the library's launchers (the same ones the separate entry points use, with
// the same launch options), so its results are theirs.
#include "internal.cuh"

using namespace retina;

struct retina_pipeline {
    retina_pipeline_config cfg;
    int device = 0;
    cudaStream_t side = nullptr;  // the search branch, highest priority
    cudaEvent_t fork = nullptr, join = nullptr;
    float4 *sorted = nullptr, *boxes = nullptr;
    int64_t *seed_offsets = nullptr;
    float *theta = nullptr, *R = nullptr;
    uint8_t *status = nullptr;
    int32_t *search_ws = nullptr;
    float *Rgrid = nullptr, *partials = nullptr;
    size_t partials_bytes = 0;
    int32_t *max_idx = nullptr, *n_max = nullptr, *maxima_ws = nullptr;
    float *max_theta = nullptr, *max_R = nullptr;
};

namespace {

bool finite_pos(float v) { return isfinite(v) && v > 0.f; }

bool valid_grid(const retina_grid &g) {
    for (int a = 0; a < 2; ++a) {
        if (!isfinite(g.lo[a]) || !finite_pos(g.step[a]) || g.n[a] <= 0) return false;
        if (!isfinite(g.lo[a] + (float)g.n[a] * g.step[a])) return false;
    }
    return true;
}

bool valid_config(const retina_pipeline_config &c) {
    if (c.model != RETINA_TOY2D && c.model != RETINA_VELO_SLOPES) return false;
    if (!valid_grid(c.grid) || !finite_pos(c.sigma_grid) || isnan(c.R0) || !finite_pos(c.merge_cells)) return false;
    for (int a = 0; a < 2; ++a)
        if ((double)c.grid.n[a] / (double)c.merge_cells > 32768.0) return false;
    const retina_ls_opts &o = c.opts;
    if (o.q < 1 || o.q > RETINA_MAX_Q) return false;
    for (int j = 0; j < o.q; ++j)
        if (!finite_pos(o.sigma[j])) return false;
    if (!(o.c1 >= 0.f && o.c1 < 1.f) || o.max_halvings < 0 || o.max_halvings > 30 || !(o.step_cap_cells > 0.f))
        return false;
    if (o.update < RETINA_UPDATE_TRUNCATED_NEWTON || o.update > RETINA_UPDATE_MODIFIED_NEWTON) return false;
    if (c.max_events < 1 || c.max_hits < 0 || c.max_tracks < 1) return false;
    if (c.seeds_per_event < 1 || c.seeds_per_event > RETINA_MAX_EXTRACT_POINTS) return false;
    if (c.max_maxima < 1 || c.max_maxima > RETINA_MAX_EXTRACT_POINTS) return false;
    return true;
}

template <typename T>
cudaError_t alloc(T *&p, size_t bytes) {
    void *v = nullptr;
    const cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 256);
    p = static_cast<T *>(v);
    return e;
}

size_t partials_needed(const retina_pipeline_config &c, int n_events) {
    const GridPlan pl = plan_grid(n_events, c.model, &c.grid, RETINA_GRID_AUTO, option_value(RETINA_OPT_GRID_SPLITS));
    return grid_partials_bytes(pl, n_events, &c.grid);
}

}  // namespace

extern "C" {

int retina_pipeline_destroy(retina_pipeline *p) {
    if (!p) return RETINA_EINVAL;
    void *bufs[] = {p->sorted, p->boxes, p->seed_offsets, p->theta, p->R, p->status, p->search_ws, p->Rgrid,
                    p->partials, p->max_idx, p->n_max, p->maxima_ws, p->max_theta, p->max_R};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->side) cudaStreamDestroy(p->side);
    delete p;
    return RETINA_OK;
}

int retina_pipeline_create(const retina_pipeline_config *config, retina_pipeline **out) {
    if (!config || !out) return RETINA_EINVAL;
    *out = nullptr;
    if (!valid_config(*config)) return RETINA_EINVAL;
    retina_pipeline *p = new retina_pipeline;
    p->cfg = *config;
    const retina_pipeline_config &c = p->cfg;
    const int64_t E = c.max_events, S = c.seeds_per_event, Km = c.max_maxima;
    const size_t cells = (size_t)c.grid.n[0] * (size_t)c.grid.n[1];
    size_t part = 0;
    for (int n = 1; n <= c.max_events; ++n) part = part > partials_needed(c, n) ? part : partials_needed(c, n);
    p->partials_bytes = part;
    int least = 0, greatest = 0;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = alloc(p->sorted, (size_t)c.max_hits * sizeof(float4));
    if (e == cudaSuccess) e = alloc(p->boxes, (size_t)prepared_box_count(c.max_hits, c.max_events) * 2 * sizeof(float4));
    if (e == cudaSuccess) e = alloc(p->seed_offsets, (size_t)(E + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = alloc(p->theta, (size_t)(E * S) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(p->R, (size_t)(E * S) * sizeof(float));
    if (e == cudaSuccess) e = alloc(p->status, (size_t)(E * S));
    if (e == cudaSuccess) e = alloc(p->search_ws, batched_ws_bytes(c.max_events));
    if (e == cudaSuccess) e = alloc(p->Rgrid, (size_t)E * cells * sizeof(float));
    if (e == cudaSuccess) e = alloc(p->partials, part);
    if (e == cudaSuccess) e = alloc(p->max_idx, (size_t)(E * Km) * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc(p->max_theta, (size_t)(E * Km) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(p->max_R, (size_t)(E * Km) * sizeof(float));
    if (e == cudaSuccess) e = alloc(p->n_max, (size_t)E * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc(p->maxima_ws, maxima_ws_bytes(c.max_events, &c.grid));
    if (e == cudaSuccess) {
        int64_t *h = new int64_t[E + 1];
        for (int64_t i = 0; i <= E; ++i) h[i] = i * S;
        e = cudaMemcpy(p->seed_offsets, h, (size_t)(E + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
        delete[] h;
    }
    if (e != cudaSuccess) {
        retina_pipeline_destroy(p);
        return RETINA_ECUDA;
    }
    *out = p;
    return RETINA_OK;
}

int retina_pipeline_run(retina_pipeline *p, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                        int32_t n_events, const float *seeds, float *grid_tracks, float *grid_track_R,
                        int32_t *grid_n_tracks, float *search_tracks, float *search_track_R,
                        int32_t *search_n_tracks, void *stream) {
    if (!p) return RETINA_EINVAL;
    const retina_pipeline_config &c = p->cfg;
    if (n_events < 0 || n_events > c.max_events || n_hits < 0 || n_hits > c.max_hits) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !seeds || !grid_tracks || !grid_track_R || !grid_n_tracks || !search_tracks ||
        !search_track_R || !search_n_tracks)
        return RETINA_EINVAL;
    if (n_hits > 0 && (!hits || ((uintptr_t)hits & 15u))) return RETINA_EINVAL;
    if ((uintptr_t)seeds & 7u) return RETINA_EINVAL;
    const GridPlan plan = plan_grid(n_events, c.model, &c.grid, RETINA_GRID_AUTO, option_value(RETINA_OPT_GRID_SPLITS));
    if (grid_partials_bytes(plan, n_events, &c.grid) > p->partials_bytes) return RETINA_ENOSPACE;
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t S = c.seeds_per_event, n_seeds = (int64_t)n_events * S;
    const float4 *h4 = reinterpret_cast<const float4 *>(hits);

    cudaError_t err = launch_prepare_hits(h4, n_hits, event_offsets, n_events, c.model, p->sorted, p->boxes, st);
    if (err == cudaSuccess) err = cudaEventRecord(p->fork, st);
    if (err != cudaSuccess) return RETINA_ECUDA;
    // search branch on the pipeline's high-priority stream
    cudaError_t err2 = cudaStreamWaitEvent(p->side, p->fork, 0);
    if (err2 == cudaSuccess)
        err2 = launch_batched_search(p->sorted, n_hits, event_offsets, p->boxes, n_events, c.model, seeds, n_seeds,
                                     p->seed_offsets, nullptr, &c.opts, &c.grid, p->theta, p->R, p->status, nullptr,
                                     p->search_ws, option_value(RETINA_OPT_BATCH_SEEDS_PER_WARP),
                                     option_value(RETINA_OPT_BATCH_WARPS), option_value(RETINA_OPT_BATCH_SMEM_HITS),
                                     option_value(RETINA_OPT_BATCH_CTAS), p->side);
    if (err2 == cudaSuccess)
        err2 = launch_extract_tracks(p->theta, p->R, p->status, nullptr, n_events, (int)S, &c.grid, c.R0,
                                     c.merge_cells, search_tracks, search_track_R, nullptr, search_n_tracks,
                                     c.max_tracks, p->side);
    const cudaError_t joined = cudaEventRecord(p->join, p->side);
    // grid branch on the caller's stream
    err = launch_grid_response(plan, p->sorted, n_hits, event_offsets, p->boxes, n_events, c.model, &c.grid,
                               c.sigma_grid, p->Rgrid, p->partials, st);
    if (err == cudaSuccess)
        err = launch_grid_maxima(p->Rgrid, n_events, &c.grid, c.R0, p->max_idx, p->max_theta, p->max_R, p->n_max,
                                 c.max_maxima, p->maxima_ws, st);
    if (err == cudaSuccess)
        err = launch_extract_tracks(p->max_theta, p->max_R, nullptr, p->n_max, n_events, c.max_maxima, &c.grid,
                                    c.R0, c.merge_cells, grid_tracks, grid_track_R, nullptr, grid_n_tracks,
                                    c.max_tracks, st);
    const cudaError_t waited = joined == cudaSuccess ? cudaStreamWaitEvent(st, p->join, 0) : joined;
    return (err == cudaSuccess && err2 == cudaSuccess && waited == cudaSuccess) ? RETINA_OK : RETINA_ECUDA;
}

}  // extern "C"
