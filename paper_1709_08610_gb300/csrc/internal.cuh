// Launchers shared between the translation units of the library (internal).
#pragma once

#include "common.cuh"

namespace retina {

struct GridPlan {
    int separable;
    int tc;     // separable contraction on the tensor cores
    int tc_bn;  // its tiles' theta_1 cells: 256 when the tiles fill the GPU, else 128
    int splits;
    int tiles0, tiles1;
};
GridPlan plan_grid(int n_events, int model, const retina_grid *g, int flags, int forced_splits);
size_t grid_partials_bytes(const GridPlan &p, int n_events, const retina_grid *g);
cudaError_t launch_grid_response(const GridPlan &p, const float4 *hits, int64_t n_hits, const int64_t *off,
                                 const float4 *boxes, int n_events, int model, const retina_grid *g, float sigma, float *R, float *partials,
                                 cudaStream_t st);
size_t maxima_ws_bytes(int n_events, const retina_grid *g);
size_t maxima_ordered_ws_bytes(int n_events, const retina_grid *g);
cudaError_t launch_grid_maxima_ordered(const float *R, int n_events, const retina_grid *g, float R0,
                                       int32_t *max_idx, float *max_theta, float *max_R, int32_t *n_max, int K,
                                       int32_t *ws_counts, cudaStream_t st);
cudaError_t launch_grid_maxima(const float *R, int n_events, const retina_grid *g, float R0, int32_t *max_idx,
                               float *max_theta, float *max_R, int32_t *n_max, int K, int32_t *ws_counts,
                               cudaStream_t st);
cudaError_t launch_local_search(const float4 *hits, int64_t n_hits, const int64_t *off, const float4 *boxes,
                                int n_events, int model, const float *seeds, int n_seeds, const retina_ls_opts *o, const retina_grid *box,
                                float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals, int seeds_per_warp,
                                int warps, int smem_hits,
                                cudaStream_t st);
cudaError_t launch_response(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                            const float *theta, int n_points, float sigma, int want_derivs, float *out,
                            cudaStream_t st);
// ws: the workspace of events with more than RETINA_MAX_EXTRACT_POINTS points
// (extract_ws_stride bytes per event; ignored below that).
cudaError_t launch_extract_tracks(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                                  int n_events, int n_points, const retina_grid *box, float R0, float merge_cells,
                                  float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int K,
                                  cudaStream_t st, void *ws = nullptr);
size_t extract_ws_stride(int n_points, int dims);

cudaError_t launch_batched_search(const float4 *hits, int64_t n_hits, const int64_t *hit_off, const float4 *boxes,
                                  int n_events, int model,
                                  const float *seeds, int64_t n_seeds, const int64_t *seed_off, const int32_t *order,
                                  const retina_ls_opts *o, const retina_grid *box, float *theta_out, float *R_out,
                                  uint8_t *status, uint8_t *n_evals, int32_t *counters, int seeds_per_warp, int warps,
                                  int smem_hits, int ctas, cudaStream_t st);
cudaError_t launch_refine_maxima(const float4 *hits, int64_t n_hits, const int64_t *hit_off, const float4 *boxes,
                                 int n_events, int model, const float *theta_c, const int32_t *n_max, int K,
                                 const retina_ls_opts *o, const retina_grid *box, float *theta_out, float *R_out,
                                 uint8_t *status, int32_t *counters, int seeds_per_warp, int warps, int smem_hits,
                                 int ctas, cudaStream_t st);
size_t batched_ws_bytes(int n_events);
cudaError_t launch_local_search4(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events,
                                 const float *seeds, int n_seeds, const int32_t *seed_count, const retina_ls4_opts *o,
                                 float *theta_out, float *R_out, uint8_t *status, int smem_hits, cudaStream_t st);
int64_t prepared_box_count(int64_t n_hits, int n_events);
cudaError_t launch_pair_seeds4(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events,
                               const float *layer_z, int n_pairs, float dz_tol, float d_max, float zc_lo, float zc_hi,
                               float zref, float *seeds, int32_t *n_seeds, int K, cudaStream_t st);
cudaError_t launch_prepare_hits(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, int model,
                                float4 *sorted, float4 *boxes, cudaStream_t st);
int maxima_blocks(const retina_grid *g);
cudaError_t launch_sort_seeds(const float *seeds, int64_t n_seeds, const int64_t *off, int n_events,
                              const retina_grid *box, float *out, int32_t *perm, cudaStream_t st);
int sm_count();
int max_dynamic_smem();
cudaError_t ensure_dynamic_smem(const void *func, size_t bytes);
unsigned long long *work_counters();
int32_t *device_error_flag();
int option_value(int option);
cudaError_t launch_conv2_head_tc(const uint16_t *h1, int n_events, const float *params, uint16_t *h2, float *logits,
                                 int32_t *err, cudaStream_t st);
void count_launches(int n);
size_t extract_smem_bytes(int n_points, int dims);
cudaError_t launch_extract_tracks4(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                                   int n_events,
                                   int n_points, const retina_grid *slope_box, const float unit[4], float R0,
                                   float merge_units, float *tracks, float *track_R, int32_t *track_src,
                                   int32_t *n_tracks, int K, cudaStream_t st);

// A launch configuration that carries the stream's priority as a launch
// attribute, so that a CUDA graph captured from the stream keeps it on the
// kernel node, and optionally programmatic stream serialization (the kernel
// calls pdl_wait before reading its predecessor's output).  Use in place
// (cfg.attrs points into the object).
struct PrioLaunch {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    PrioLaunch(dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl = false) {
        int prio = 0;
        if (cudaStreamGetPriority(st, &prio) != cudaSuccess) prio = 0;
        cfg = cudaLaunchConfig_t{};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        attr[0].id = cudaLaunchAttributePriority;
        attr[0].val.priority = prio;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 2 : 1;
    }
    PrioLaunch(const PrioLaunch &) = delete;
    PrioLaunch &operator=(const PrioLaunch &) = delete;
};

// learned seed proposer
cudaError_t launch_slope_hist(const float4 *hits, int64_t n_hits, const int64_t *off, int n_events, float lo, float hi,
                              float zmin, uint16_t *feat, int32_t *counts, cudaStream_t st);
cudaError_t launch_seednet_forward(const uint16_t *feat, int n_events, const float *params, float *logits,
                                   uint16_t *h1, uint16_t *h2, cudaStream_t st);
size_t seednet_train_ws_bytes(int n_events);
cudaError_t launch_seednet_train_step(const uint16_t *feat, const uint8_t *labels, int n_events, float *params,
                                      float *m, float *v, int step, float lr, float b1, float b2, float eps,
                                      float *loss_out, float *grad_out, void *ws, cudaStream_t st);
cudaError_t launch_seednet_adam(float *params, float *m, float *v, const float *grad, int step, float lr, float b1,
                                float b2, float eps, cudaStream_t st);
cudaError_t launch_propose_seeds(const float *logits, int n_events, int K, float lo, float hi, float zmin, int n_min,
                                 const float4 *hits, int64_t n_hits, const int64_t *off, float *seeds, int32_t *idx,
                                 cudaStream_t st);

}  // namespace retina
