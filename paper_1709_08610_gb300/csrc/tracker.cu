// Native executor of Algorithm 1 over a batch of events (retina_tracker_*):
// hit ordering, the starting points (the learned proposer, or the caller's),
// their spatial order, the persistent batched search and cluster / select,
// recorded once per event count as a CUDA graph and replayed.  The tracker
// owns its input and output buffers, so a run is either a replay on those
// buffers (retina_tracker_step) or host copies in, a replay and host copies
// out, all enqueued on the caller's stream (retina_tracker_run_host).
// Creation validates the configuration and allocates every buffer; runs
// allocate nothing.  The launchers are the library's own, with the same
// arguments the separate entry points pass, so results are theirs.
#include <cstring>

#include "internal.cuh"

using namespace retina;

namespace {

struct GraphKey {
    int n_events = -1, spw = 0, warps = 0, smem_hits = 0, ctas = 0, seednet_tc = 0;
    bool operator==(const GraphKey &o) const {
        return n_events == o.n_events && spw == o.spw && warps == o.warps && smem_hits == o.smem_hits &&
               ctas == o.ctas && seednet_tc == o.seednet_tc;
    }
};

}  // namespace

struct retina_tracker {
    retina_tracker_config cfg;
    bool learned = false;
    int device = 0;
    cudaStream_t cap = nullptr;  // capture stream (graphs cannot be recorded on a legacy stream)
    // run_host's hit copy: on its own stream, after the previous step's hit
    // ordering (the one launch that reads the unsorted hits) - not after the
    // whole previous step - so it overlaps that step's search
    cudaStream_t copy = nullptr;
    cudaEvent_t hits_free = nullptr, hits_in = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    cudaEvent_t marks[RETINA_TRACKER_MARKS] = {};  // stage marks (retina_tracker_set_marks)
    bool marked = false;
    // inputs
    float4 *hits = nullptr;
    int64_t *offsets = nullptr;
    float *seeds = nullptr;
    // intermediates
    float4 *sorted = nullptr, *boxes = nullptr;
    float *seeds_sorted = nullptr;
    int64_t *seed_offsets = nullptr;
    float *params = nullptr, *logits = nullptr;
    uint16_t *feat = nullptr, *h1 = nullptr;
    float *theta = nullptr, *R = nullptr;
    uint8_t *status = nullptr;
    int32_t *counters = nullptr;
    // outputs
    float *tracks = nullptr, *track_R = nullptr;
    int32_t *n_tracks = nullptr;
};

namespace {

bool finite_pos(float v) { return isfinite(v) && v > 0.f; }

bool valid_config(const retina_tracker_config &c) {
    for (int a = 0; a < 2; ++a) {
        if (!isfinite(c.box.lo[a]) || !finite_pos(c.box.step[a]) || c.box.n[a] <= 0) return false;
        if (!isfinite(c.box.lo[a] + (float)c.box.n[a] * c.box.step[a])) return false;
        if ((double)c.box.n[a] / (double)c.merge_cells > 32768.0) return false;
    }
    if (isnan(c.R0) || !finite_pos(c.merge_cells)) return false;
    const retina_ls_opts &o = c.opts;
    if (o.q < 1 || o.q > RETINA_MAX_Q) return false;
    for (int j = 0; j < o.q; ++j)
        if (!finite_pos(o.sigma[j])) return false;
    if (!(o.c1 >= 0.f && o.c1 < 1.f) || o.max_halvings < 0 || o.max_halvings > 30 || !(o.step_cap_cells > 0.f))
        return false;
    if (o.update < RETINA_UPDATE_TRUNCATED_NEWTON || o.update > RETINA_UPDATE_MODIFIED_NEWTON) return false;
    if (c.max_events < 1 || c.max_events > 65535 || c.max_hits < 0 || c.max_tracks < 1) return false;
    if (c.seeds_per_event < 1 || c.seeds_per_event > RETINA_MAX_EXTRACT_POINTS) return false;
    if (c.sort_seeds != 0 && c.sort_seeds != 1) return false;
    if (c.seeds_per_warp != 0 && c.seeds_per_warp != 1 && c.seeds_per_warp != 2 && c.seeds_per_warp != 4)
        return false;
    if (c.warps != 0 && c.warps != 8 && c.warps != 16 && c.warps != 32) return false;
    if (c.smem_hits < 0 || c.smem_hits > 12288 || c.ctas < 0 || c.ctas > (1 << 20)) return false;
    return true;
}

template <typename T>
cudaError_t alloc(T *&p, size_t bytes) {
    void *v = nullptr;
    const cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 256);
    p = static_cast<T *>(v);
    return e;
}

// The launch shape the next run uses: the configuration's, else the option in force.
GraphKey current_key(const retina_tracker &t, int n_events) {
    const retina_tracker_config &c = t.cfg;
    GraphKey k;
    k.n_events = n_events;
    k.spw = c.seeds_per_warp ? c.seeds_per_warp : option_value(RETINA_OPT_BATCH_SEEDS_PER_WARP);
    k.warps = c.warps ? c.warps : option_value(RETINA_OPT_BATCH_WARPS);
    k.smem_hits = c.smem_hits ? c.smem_hits : option_value(RETINA_OPT_BATCH_SMEM_HITS);
    k.ctas = c.ctas ? c.ctas : option_value(RETINA_OPT_BATCH_CTAS);
    k.seednet_tc = option_value(RETINA_OPT_SEEDNET_TC);
    return k;
}

// Record stage mark i on st: as an event node of the graph while capturing.
cudaError_t mark(const retina_tracker &t, int i, cudaStream_t st, bool capturing) {
    if (!t.marked) return cudaSuccess;
    return capturing ? cudaEventRecordWithFlags(t.marks[i], st, cudaEventRecordExternal) : cudaEventRecord(t.marks[i], st);
}

// Every launch of one step on the tracker's buffers.  n_hits is the capacity:
// the event offsets bound every read, so one recording serves any batch that
// fits.
cudaError_t enqueue_step(retina_tracker &t, const GraphKey &k, cudaStream_t st, bool capturing) {
    const retina_tracker_config &c = t.cfg;
    const int E = k.n_events;
    const int64_t H = c.max_hits, S = c.seeds_per_event, n_seeds = (int64_t)E * S;
    const float lo = -0.5f, hi = 0.5f, zmin = 50.f;  // the proposer's histogram (as trained)
    cudaError_t err = mark(t, 0, st, capturing);
    if (err == cudaSuccess) err = launch_prepare_hits(t.hits, H, t.offsets, E, RETINA_VELO_SLOPES, t.sorted, t.boxes, st);
    // every later launch reads the ordered copy: the input buffer is free
    // (the proposer's histogram and sub-cell sums are integer counts and
    // fixed-point sums, the same in any hit order)
    if (err == cudaSuccess)
        err = capturing ? cudaEventRecordWithFlags(t.hits_free, st, cudaEventRecordExternal)
                        : cudaEventRecord(t.hits_free, st);
    if (err == cudaSuccess) err = mark(t, 1, st, capturing);
    if (err == cudaSuccess && t.learned) {
        err = launch_slope_hist(t.sorted, H, t.offsets, E, lo, hi, zmin, t.feat, nullptr, st);
        if (err == cudaSuccess) err = launch_seednet_forward(t.feat, E, t.params, t.logits, t.h1, nullptr, st);
        if (err == cudaSuccess)
            err = launch_propose_seeds(t.logits, E, (int)S, lo, hi, zmin, 3, t.sorted, H, t.offsets, t.seeds, nullptr,
                                       st);
    }
    if (err == cudaSuccess) err = mark(t, 2, st, capturing);
    const float *seeds = t.seeds;
    if (err == cudaSuccess && c.sort_seeds) {
        err = launch_sort_seeds(t.seeds, n_seeds, t.seed_offsets, E, &c.box, t.seeds_sorted, nullptr, st);
        seeds = t.seeds_sorted;
    }
    if (err == cudaSuccess) err = mark(t, 3, st, capturing);
    if (err == cudaSuccess)
        err = launch_batched_search(t.sorted, H, t.offsets, t.boxes, E, RETINA_VELO_SLOPES, seeds, n_seeds,
                                    t.seed_offsets, nullptr, &c.opts, &c.box, t.theta, t.R, t.status, nullptr,
                                    t.counters, k.spw, k.warps, k.smem_hits, k.ctas, st);
    if (err == cudaSuccess) err = mark(t, 4, st, capturing);
    if (err == cudaSuccess)
        err = launch_extract_tracks(t.theta, t.R, t.status, nullptr, E, (int)S, &c.box, c.R0, c.merge_cells, t.tracks,
                                    t.track_R, nullptr, t.n_tracks, c.max_tracks, st);
    if (err == cudaSuccess) err = mark(t, 5, st, capturing);
    return err;
}

// Replay (recording first when the event count or the launch shape changed).
int step(retina_tracker &t, int n_events, cudaStream_t st) {
    const GraphKey k = current_key(t, n_events);
    if (!t.cfg.use_graph) return enqueue_step(t, k, st, false) == cudaSuccess ? RETINA_OK : RETINA_ECUDA;
    if (!t.exec || !(t.key == k)) {
        if (t.exec) {
            cudaGraphExecDestroy(t.exec);
            t.exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t err = cudaStreamBeginCapture(t.cap, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return RETINA_ECUDA;
        const cudaError_t lerr = enqueue_step(t, k, t.cap, true);
        err = cudaStreamEndCapture(t.cap, &g);
        if (lerr != cudaSuccess || err != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return RETINA_ECUDA;
        }
        err = cudaGraphInstantiate(&t.exec, g, 0);
        cudaGraphDestroy(g);
        if (err != cudaSuccess) {
            t.exec = nullptr;
            return RETINA_ECUDA;
        }
        t.key = k;
    }
    return cudaGraphLaunch(t.exec, st) == cudaSuccess ? RETINA_OK : RETINA_ECUDA;
}

}  // namespace

extern "C" {

int retina_tracker_destroy(retina_tracker *t) {
    if (!t) return RETINA_EINVAL;
    if (t->exec) cudaGraphExecDestroy(t->exec);
    void *bufs[] = {t->hits,  t->offsets, t->seeds, t->sorted, t->boxes,  t->seeds_sorted, t->seed_offsets,
                    t->params, t->logits, t->feat,  t->h1,     t->theta,  t->R,            t->status,
                    t->counters, t->tracks, t->track_R, t->n_tracks};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (t->cap) cudaStreamDestroy(t->cap);
    if (t->copy) cudaStreamDestroy(t->copy);
    if (t->hits_free) cudaEventDestroy(t->hits_free);
    if (t->hits_in) cudaEventDestroy(t->hits_in);
    delete t;
    return RETINA_OK;
}

int retina_tracker_create(const retina_tracker_config *config, const float *seednet_params, retina_tracker **out) {
    if (!config || !out) return RETINA_EINVAL;
    *out = nullptr;
    if (!valid_config(*config)) return RETINA_EINVAL;
    retina_tracker *t = new retina_tracker;
    t->cfg = *config;
    t->learned = seednet_params != nullptr;
    const retina_tracker_config &c = t->cfg;
    const int64_t E = c.max_events, S = c.seeds_per_event, H = c.max_hits, K = c.max_tracks;
    const int64_t px = E * RETINA_SEEDNET_BINS * RETINA_SEEDNET_BINS;
    cudaError_t e = cudaGetDevice(&t->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->hits_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->hits_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = alloc(t->hits, (size_t)H * sizeof(float4));
    if (e == cudaSuccess) e = alloc(t->offsets, (size_t)(E + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = alloc(t->seeds, (size_t)(E * S) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->sorted, (size_t)H * sizeof(float4));
    if (e == cudaSuccess) e = alloc(t->boxes, (size_t)prepared_box_count(H, (int)E) * 2 * sizeof(float4));
    if (e == cudaSuccess && c.sort_seeds) e = alloc(t->seeds_sorted, (size_t)(E * S) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->seed_offsets, (size_t)(E + 1) * sizeof(int64_t));
    if (e == cudaSuccess && t->learned) {
        e = alloc(t->params, (size_t)RETINA_SEEDNET_PARAMS * sizeof(float));
        if (e == cudaSuccess) e = alloc(t->logits, (size_t)px * sizeof(float));
        if (e == cudaSuccess) e = alloc(t->feat, (size_t)px * sizeof(uint16_t));
        if (e == cudaSuccess) e = alloc(t->h1, (size_t)px * 16 * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(t->params, seednet_params, (size_t)RETINA_SEEDNET_PARAMS * sizeof(float),
                           cudaMemcpyDefault);
    }
    if (e == cudaSuccess) e = alloc(t->theta, (size_t)(E * S) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->R, (size_t)(E * S) * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->status, (size_t)(E * S));
    if (e == cudaSuccess) e = alloc(t->counters, batched_ws_bytes((int)E));
    if (e == cudaSuccess) e = alloc(t->tracks, (size_t)(E * K) * 2 * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->track_R, (size_t)(E * K) * sizeof(float));
    if (e == cudaSuccess) e = alloc(t->n_tracks, (size_t)E * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(t->offsets, 0, (size_t)(E + 1) * sizeof(int64_t));
    if (e == cudaSuccess) {
        int64_t *h = new int64_t[E + 1];
        for (int64_t i = 0; i <= E; ++i) h[i] = i * S;
        e = cudaMemcpy(t->seed_offsets, h, (size_t)(E + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
        delete[] h;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        retina_tracker_destroy(t);
        return RETINA_ECUDA;
    }
    *out = t;
    return RETINA_OK;
}

int retina_tracker_buffers(retina_tracker *t, float **hits, int64_t **event_offsets, float **seeds, float **tracks,
                           float **track_R, int32_t **n_tracks) {
    if (!t) return RETINA_EINVAL;
    if (hits) *hits = reinterpret_cast<float *>(t->hits);
    if (event_offsets) *event_offsets = t->offsets;
    if (seeds) *seeds = t->seeds;
    if (tracks) *tracks = t->tracks;
    if (track_R) *track_R = t->track_R;
    if (n_tracks) *n_tracks = t->n_tracks;
    return RETINA_OK;
}

int retina_tracker_set_marks(retina_tracker *t, void *const *events, int32_t n) {
    if (!t || (n != 0 && n != RETINA_TRACKER_MARKS) || (n && !events)) return RETINA_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!events[i]) return RETINA_EINVAL;
    for (int i = 0; i < RETINA_TRACKER_MARKS; ++i) t->marks[i] = n ? (cudaEvent_t)events[i] : nullptr;
    t->marked = n != 0;
    if (t->exec) {  // the recorded graph has (or lacks) the old marks: record again at the next step
        cudaGraphExecDestroy(t->exec);
        t->exec = nullptr;
    }
    return RETINA_OK;
}

int retina_tracker_step(retina_tracker *t, int32_t n_events, void *stream) {
    if (!t || n_events < 0 || n_events > t->cfg.max_events) return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    return step(*t, n_events, (cudaStream_t)stream);
}

int retina_tracker_run_host(retina_tracker *t, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                            int32_t n_events, const float *seeds, float *tracks, float *track_R, int32_t *n_tracks,
                            void *stream) {
    if (!t || n_events < 0 || n_events > t->cfg.max_events || n_hits < 0 || n_hits > t->cfg.max_hits)
        return RETINA_EINVAL;
    if (n_events == 0) return RETINA_OK;
    if (!event_offsets || !tracks || !track_R || !n_tracks || (n_hits > 0 && !hits)) return RETINA_EINVAL;
    if (!t->learned && !seeds) return RETINA_EINVAL;
    // the offsets must describe events inside the copied hits (the device clamps
    // them anyway; a malformed batch is refused before anything is enqueued)
    for (int32_t e = 0; e <= n_events; ++e) {
        const int64_t v = event_offsets[e];
        if (v < 0 || v > n_hits || (e > 0 && v < event_offsets[e - 1])) return RETINA_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const retina_tracker_config &c = t->cfg;
    const size_t S = (size_t)c.seeds_per_event, K = (size_t)c.max_tracks;
    // the hits on the copy stream, once the previous step's hit ordering is
    // done (a wait on a never-recorded event passes); the step waits for them
    cudaError_t err = cudaStreamWaitEvent(t->copy, t->hits_free, 0);
    if (err == cudaSuccess && n_hits > 0)
        err = cudaMemcpyAsync(t->hits, hits, (size_t)n_hits * sizeof(float4), cudaMemcpyHostToDevice, t->copy);
    if (err == cudaSuccess) err = cudaEventRecord(t->hits_in, t->copy);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, t->hits_in, 0);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(t->offsets, event_offsets, (size_t)(n_events + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && !t->learned)
        err = cudaMemcpyAsync(t->seeds, seeds, (size_t)n_events * S * 2 * sizeof(float), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return RETINA_ECUDA;
    const int rc = step(*t, n_events, st);
    if (rc != RETINA_OK) return rc;
    err = cudaMemcpyAsync(n_tracks, t->n_tracks, (size_t)n_events * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(tracks, t->tracks, (size_t)n_events * K * 2 * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(track_R, t->track_R, (size_t)n_events * K * sizeof(float), cudaMemcpyDeviceToHost, st);
    return err == cudaSuccess ? RETINA_OK : RETINA_ECUDA;
}

}  // extern "C"
