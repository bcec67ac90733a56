/*
 * retina.h - C ABI of the GB300 (sm_103a) Artificial Retina library.
 *
 * The library evaluates the retina response of arXiv:1709.08610 (Borisyak,
 * Ustyuzhanin, Derkach, Belous, "Numerical optimization for Artificial
 * Retina Algorithm"), Section 2, Eq. 1:
 *
 *     R(theta) = sum_k exp(-s(x_k, theta)^2 / sigma^2)
 *
 * over all hits x_k of an event, on a grid of units (Eq. 2, the brute-force
 * grid algorithm of Section 2) or along a multistart truncated-Newton local
 * search (Algorithm 1 with the update and sigma schedule of Section 3), and
 * turns grid maxima or converged points into tracks (the cluster / select
 * lines of Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller (allocated
 *   with cudaMalloc or any allocator of device memory); the library never
 *   frees them, never retains them after the call returns, and allocates no
 *   device memory itself.  Scratch memory comes from a caller-provided
 *   workspace whose size the matching *_workspace_size function reports.
 *   Struct arguments (retina_grid, retina_ls_opts) are HOST pointers, read
 *   during the call only.
 * - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *   NULL means the legacy default stream).  Outputs are valid once the
 *   stream reaches the call.
 * - Return value: RETINA_OK or an error code.  Arguments are validated on
 *   the host before any launch; on RETINA_EINVAL nothing was launched.
 *   RETINA_ECUDA reports a failed launch (cudaGetLastError).  Conditions
 *   found on the device (a non-finite point, an output list that overflowed)
 *   are written to status arrays and counts; kernels never trap.
 * - hits: float32 [n_hits][4], 16-byte aligned, events concatenated:
 *   event e owns rows event_offsets[e] .. event_offsets[e+1]-1
 *   (event_offsets: int64 [n_events + 1], non-decreasing, device memory).
 *   Kernels clamp every offset to [0, n_hits] and treat a decreasing pair as
 *   an empty event, so malformed offsets cannot make them read outside hits.
 *   boxes: nullable; when given, hits must be the output of
 *   retina_prepare_hits (each event's hits in its spatial order) and boxes
 *   its block boxes.  The kernels then skip, per point or per tile, every
 *   block of 32 hits whose terms of Eq. 1 are all exactly zero in float32,
 *   so the results are bitwise those of evaluating every hit in that order.
 *   Row layout per model:
 *     RETINA_TOY2D       (x, y, -, -): 2D line y = theta0 * x + theta1 seen by
 *                        detector planes x = const; s = y - theta0 x - theta1
 *                        (Section 2, Figure 1 caption).
 *     RETINA_VELO_SLOPES (x, y, z, -): straight 3D track through the origin
 *                        with slopes theta = (t_x, t_y); s is the distance in
 *                        the layer z = const between the hit and the track's
 *                        crossing (t_x z, t_y z) (Section 3).
 * - A grid / box: cell centres theta_a = lo[a] + (i_a + 1/2) step[a],
 *   i_a = 0 .. n[a]-1; the box is [lo, lo + n * step).  Response grids are
 *   float32 [n_events][n[1]][n[0]] (theta1 slow, theta0 fast), and a cell's
 *   linear index is i1 * n[0] + i0.
 */
#ifndef RETINA_H
#define RETINA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RETINA_OK 0
#define RETINA_EINVAL 1   /* invalid argument; nothing launched               */
#define RETINA_ECUDA 2    /* a CUDA launch or runtime call failed             */
#define RETINA_ENOSPACE 3 /* workspace too small, or a size limit exceeded    */

#define RETINA_TOY2D 0
#define RETINA_VELO_SLOPES 1

/* grid-scan method flags (retina_grid_scan `flags`) */
#define RETINA_GRID_AUTO 0
#define RETINA_GRID_DIRECT 1    /* force the per-pair exp kernel           */
#define RETINA_GRID_SEPARABLE 2 /* force exp(-u^2-v^2)=exp(-u^2)exp(-v^2)   */
#define RETINA_GRID_TENSOR 3    /* the separable contraction on the tcgen05
                                   tensor cores (3 x TF32 split products)    */
                                /* contraction (RETINA_VELO_SLOPES only)     */

/* maximum number of local-search updates q */
#define RETINA_MAX_Q 8
/* maximum number of candidate points per event in retina_extract_tracks */
#define RETINA_MAX_EXTRACT_POINTS 8192

/* tuning options (retina_set_option); values are validated, defaults in () */
#define RETINA_OPT_LS_SEEDS_PER_WARP 1 /* 1, 2 or 4 seeds per warp (1)          */
#define RETINA_OPT_LS_SMEM_HITS 2      /* hits staged in shared memory (4096)   */
#define RETINA_OPT_GRID_SPLITS 3       /* hit slices per grid tile, 0=auto (0)  */
#define RETINA_OPT_LS_WARPS 4          /* warps per search CTA: 4, 8 or 16 (8)  */
#define RETINA_OPT_BATCH_SEEDS_PER_WARP 5 /* batched search: 1, 2 or 4 (1)      */
#define RETINA_OPT_BATCH_WARPS 6       /* batched search CTA warps: 8,16,32 (16) */
#define RETINA_OPT_BATCH_SMEM_HITS 7   /* batched search staged hits (8192)     */
#define RETINA_OPT_BATCH_CTAS 8        /* batched search CTAs, 0 = fill the GPU (0);
                                          fewer leave room for kernels running
                                          concurrently on other streams          */
#define RETINA_OPT_GRID_TC 10          /* RETINA_GRID_AUTO on slope-model grids
                                          picks the tensor-core contraction (1)
                                          or the CUDA-core one (0); default 1   */
#define RETINA_OPT_SEEDNET_TC 9        /* seed net's second convolution on the
                                          tcgen05 tensor cores (1) or the FP32
                                          CUDA cores (0); default 1               */

typedef struct {
    float lo[2];   /* lower edge of the box per axis                      */
    float step[2]; /* cell size per axis (> 0)                            */
    int32_t n[2];  /* cells per axis (> 0)                                */
} retina_grid;

/* Options of the local search (Algorithm 1; Section 3). */
typedef struct {
    int32_t q;            /* updates per seed, 1 .. RETINA_MAX_Q (paper: 3)     */
    float sigma[8];       /* bandwidth at update j (paper: 0.3, 0.175, 0.05)    */
    float c1;             /* Armijo sufficient-increase constant, in [0, 1)    */
    int32_t max_halvings; /* backtracking halvings after t = 1, 0 .. 30        */
    float step_cap_cells; /* cap on max_a |p_a| / step_a, > 0                  */
    int32_t update;       /* direction of each update (RETINA_UPDATE_*); 0, the */
                          /* paper's truncated Newton, when zero-initialised   */
} retina_ls_opts;

/*
 * Update directions (retina_ls_opts.update).  Section 3 reports truncated
 * Newton as the best of the methods it examined; the other two are the
 * textbook alternatives, for comparison.  All three share the step cap and
 * the Armijo backtracking.
 *   RETINA_UPDATE_TRUNCATED_NEWTON  Newton-CG (retina_local_search, step 2).
 *   RETINA_UPDATE_STEEPEST_ASCENT   p = grad R.
 *   RETINA_UPDATE_MODIFIED_NEWTON   p solves (B + tau I) p = grad R with
 *       B = -Hess R, tau = max(0, delta - mu1), mu1 <= mu2 the eigenvalues of
 *       B, delta = 1e-3 max(|mu1|, |mu2|) (Nocedal & Wright, Section 3.4);
 *       B = 0 gives p = grad R.
 */
#define RETINA_UPDATE_TRUNCATED_NEWTON 0
#define RETINA_UPDATE_STEEPEST_ASCENT 1
#define RETINA_UPDATE_MODIFIED_NEWTON 2

/* Human-readable text for a status code (static storage). */
const char *retina_strerror(int code);

/* ABI version of this header (incremented on incompatible change). */
int retina_abi_version(void);

/* Set a process-wide tuning option (RETINA_OPT_*).  Affects launches made
 * after the call; results do not depend on it beyond FP32 summation order.
 * Returns RETINA_EINVAL for an unknown option or an out-of-range value. */
int retina_set_option(int32_t option, int32_t value);
int retina_get_option(int32_t option, int32_t *value);

/* Device-side error flag of the library (on the current device): kernels set
 * it to 1 when one of their bounded waits expires (their outputs are then
 * not valid) instead of hanging or trapping.  flag (nullable, host) receives
 * it; reset = 1 clears it.  Synchronous device copies. */
int retina_device_error(int32_t *flag, int32_t reset);

/* Number of kernels this library has launched in this process (all entry
 * points, all threads); callers difference it around a region to count the
 * library's launches in it.  Not part of the paper: instrumentation. */
uint64_t retina_launch_count(void);

/* Work counters (instrumentation, not part of the paper): when enabled, the
 * response kernels add the (point or cell, hit) pairs they evaluate, after
 * block skipping, to device counters:
 *   [RETINA_WORK_GRID] grid response pairs, [RETINA_WORK_RGH] search pairs of
 *   R/grad/Hess passes, [RETINA_WORK_R] search pairs of R-only passes.
 * retina_work_counters(enable, reset, out): enable = 1 / 0 switches counting
 * on / off for later launches (-1 leaves it), reset = 1 zeroes the counters,
 * out (nullable, host, RETINA_WORK_KINDS entries) receives their values.
 * Reset and read are synchronous device copies; counting costs one atomic per
 * CTA or warp. */
#define RETINA_WORK_KINDS 4
#define RETINA_WORK_GRID 0
#define RETINA_WORK_RGH 1
#define RETINA_WORK_R 2
int retina_work_counters(int32_t enable, int32_t reset, uint64_t *out);

/*
 * retina_alu_probe - throughput probe of the arithmetic pipes the retina
 * kernels use (not part of the paper; it supplies the FP32 / SFU peaks of
 * the roofline, which no vendor table gives for this part).  Launches one
 * saturating kernel on `stream`: every thread runs `iters` iterations of
 * eight independent dependency chains of
 *   kind 0: FP32 fused multiply-add (FFMA pipe),
 *   kind 1: ex2.approx (MUFU / SFU pipe),
 *   kind 2: packed FP32x2 fused multiply-add (two FMAs per instruction).
 * *ops receives the number of FP32 operations (kind 0, 2: FMAs; kind 1:
 * ex2) the launch performs; time the launch with events on `stream`.
 * sink: float32 device buffer of retina_alu_probe_sink_floats() elements
 * (keeps the chains live).  iters in [1, 1<<20].
 */
int64_t retina_alu_probe_sink_floats(void);
int retina_alu_probe(int32_t kind, int32_t iters, float *sink, double *ops, void *stream);

/*
 * retina_prepare_hits - spatial order and block boxes for exact skipping.
 *
 * Not a step of the paper: an acceleration structure for Eq. 1.  Per event,
 * sorts the hits into a spatial order and writes them to sorted_out
 * (float32 [n_hits][4], same event offsets); block b of event e (sorted hits
 * 32 b .. 32 b + 31) gets an 8-float box in boxes_out row
 * floor(event_offsets[e] / 32) + e + b.  Order: each super-chunk of 32768
 * consecutive hits of an event is sorted by (code, index).  Slope model: code
 * = band of |z| (octaves [0,16), [16,32), ..., [512, inf) mm; NaN in the
 * last) above the Hilbert index (order 8) of the slopes (x/z, y/z) quantised
 * to 256 levels on [-1, 1] (clamped); box = (min, max of x/z, min, max of
 * y/z, min, max of |z|, 0, 0).  2D toy: code = x band above the quantised y;
 * box = (xmin, xmax, ymin, ymax, 0, 0, 0, 0).  boxes_out: float32
 * [retina_prepare_hits_box_count(n_hits, n_events)][8].  A box with a
 * non-finite value (e.g. a hit at z = 0) is infinite: never skipped.  The
 * order of hits within an event does not change R beyond float32 summation
 * order.
 */
int64_t retina_prepare_hits_box_count(int64_t n_hits, int32_t n_events);
int retina_prepare_hits(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                        int32_t model, float *sorted_out, float *boxes_out, void *stream);

/*
 * retina_grid_scan - response on a grid of units and its local maxima.
 *
 * Paper: Section 2, Eq. 2 (R_ij = R(theta_ij) for every unit) and steps 2-4
 * of the grid algorithm (compute the grid response, select activated units,
 * estimate parameters).  A unit is selected when R_ij >= R0 and it beats
 * every existing neighbour of its 3 x 3 neighbourhood in the order
 * (R, -linear index): a strict local maximum, ties going to the lower
 * linear index.  Its estimate is the cell centre.
 *
 *   hits, event_offsets, n_events, model : see the conventions above.
 *   g        : host pointer; the grid of units.
 *   sigma    : bandwidth (> 0, finite).
 *   R0       : selection threshold.
 *   flags    : RETINA_GRID_AUTO / _DIRECT / _SEPARABLE.
 *   R_out    : nullable; float32 [n_events][n1][n0] response grid.  When
 *              NULL the grid lives in the workspace.
 *   max_idx  : int32 [n_events][K]; linear cell index of each selected unit,
 *              increasing, per event.
 *   max_theta: float32 [n_events][K][2]; cell centre of each selected unit.
 *   max_R    : float32 [n_events][K]; its response.
 *   n_max    : int32 [n_events]; number of selected units (may exceed K:
 *              only the first K, in index order, are written).
 *   K        : capacity per event (>= 1).
 *   ws, ws_bytes : workspace of at least retina_grid_scan_workspace_size().
 * Returns RETINA_ENOSPACE (nothing launched) when ws_bytes is too small.
 */
int retina_grid_scan_workspace_size(int32_t n_events, int32_t model, const retina_grid *g, int32_t flags,
                                    int32_t store_R, size_t *bytes);
int retina_grid_scan(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events, int32_t model,
                     const retina_grid *g, float sigma, float R0, int32_t flags, float *R_out, int32_t *max_idx,
                     float *max_theta, float *max_R, int32_t *n_max, int32_t K, void *ws, size_t ws_bytes,
                     void *stream);

/*
 * retina_grid_response - the grid response alone (Section 2, Eq. 2): writes
 * R_out float32 [n_events][n1][n0] (required), no selection.  Same arguments
 * as retina_grid_scan; workspace from retina_grid_response_workspace_size.
 */
int retina_grid_response_workspace_size(int32_t n_events, int32_t model, const retina_grid *g, int32_t flags,
                                        size_t *bytes);
int retina_grid_response(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events,
                         int32_t model, const retina_grid *g, float sigma, int32_t flags, float *R_out, void *ws,
                         size_t ws_bytes, void *stream);

/*
 * retina_grid_maxima - the selection step alone, on a caller-supplied grid.
 *
 * Paper: Section 2, steps 3-4 of the grid algorithm.  Same rule and outputs
 * as retina_grid_scan, reading R float32 [n_events][n1][n0].
 */
int retina_grid_maxima_workspace_size(int32_t n_events, const retina_grid *g, size_t *bytes);
int retina_grid_maxima(const float *R, int32_t n_events, const retina_grid *g, float R0, int32_t *max_idx,
                       float *max_theta, float *max_R, int32_t *n_max, int32_t K, void *ws, size_t ws_bytes,
                       void *stream);

/*
 * retina_grid_maxima_static - retina_grid_maxima without a workspace.
 *
 * The paper has no counterpart: this is an interface variant for callers
 * that cannot allocate device memory - for example a plugin running inside a
 * host application whose memory manager owns every device allocation, or a
 * foreign-language caller with no device allocator of its own - and so
 * cannot supply the workspace the other entry points take.  Same rule,
 * arguments and outputs as retina_grid_maxima; the outputs are still the
 * caller's.
 *
 * Its scratch (two int32 per 2048-cell block per event) lives in one
 * library-owned device array of RETINA_STATIC_SCRATCH_BYTES, held by every
 * GPU that loads the library until the process exits.  Limits and behaviour:
 * - 2 * n_events * ceil(n0 * n1 / 2048) * 4 bytes must fit in
 *   RETINA_STATIC_SCRATCH_BYTES (1 MiB: e.g. 256 events of 1024 x 1024 or 64
 *   of 2048 x 2048); larger requests return RETINA_ENOSPACE, nothing launched.
 * - n_events above 65535 returns RETINA_EINVAL, nothing launched (as for
 *   retina_grid_maxima).
 * - The first call on a device looks up the array's device address (with that
 *   device current, i.e. the CUDA runtime's current device must be the one
 *   `stream` belongs to); make that first call before any stream capture.
 * - All calls share the one array, so calls whose kernels overlap on the GPU
 *   (different streams, no ordering between them) race and give undefined
 *   results; calls ordered on one stream are safe.  The array keeps the last
 *   call's contents, and each call writes every part it reads first, so no
 *   result depends on an earlier call.
 * - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define RETINA_STATIC_SCRATCH_BYTES (1 << 20)
int retina_grid_maxima_static(const float *R, int32_t n_events, const retina_grid *g, float R0, int32_t *max_idx,
                              float *max_theta, float *max_R, int32_t *n_max, int32_t K, void *stream);

/*
 * retina_response - R, grad R and Hess R at arbitrary points.
 *
 * Paper: Section 2, Eq. 1, and the remark that the gradient and the Hessian
 * cost little more than R itself:
 *     grad R = (2/sigma^2) sum_k e_k J_k^T r_k
 *     Hess R = sum_k e_k [(4/sigma^4)(J_k^T r_k)(J_k^T r_k)^T - (2/sigma^2) J_k^T J_k]
 * with r_k the residual of hit k and J_k its Jacobian in theta.
 *
 *   theta : float32 [n_events][n_points][2].
 *   out   : float32 [n_events][n_points][6] = (R, g0, g1, H00, H01, H11);
 *           when want_derivs == 0 only R (column 0) is written.
 */
int retina_response(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events, int32_t model,
                    const float *theta, int32_t n_points, float sigma, int32_t want_derivs, float *out,
                    void *stream);

/*
 * retina_local_search - Algorithm 1's q updates for every seed.
 *
 * Paper: Algorithm 1 (seeds drawn from a prior, q updates each using R,
 * grad R and Hess R) with the truncated Newton update and the annealed
 * bandwidths of Section 3.  Update j (j = 1..q) at bandwidth sigma_j:
 *   1. (R, g, H) at theta.
 *   2. Direction p: conjugate gradients on -H p = g from p = 0 (Newton-CG,
 *      Nocedal & Wright, Algorithm 7.1), forcing tolerance
 *      min(1/2, sqrt|g|) |g|, at most 2 iterations; on non-positive
 *      curvature of -R along the CG direction: p = g at the first
 *      iteration, else the current iterate.  (opts->update selects one of
 *      the comparison directions of RETINA_UPDATE_* instead.)
 *   3. If max_a |p_a| / step_a > step_cap_cells, p is scaled down to it.
 *   4. Backtracking: the first t in 1, 1/2, ..., 2^-max_halvings with
 *      R(theta + t p) >= R(theta) + c1 t g.p is taken; if none, theta
 *      stays and the seed's status becomes 1.
 * Then R_out = R(theta_q; sigma_q).
 *
 *   seeds     : float32 [n_events][n_seeds][2] starting points.
 *   opts      : host pointer.
 *   box       : host pointer; its step sizes set the step cap, and the box
 *               decides status 2.
 *   theta_out : float32 [n_events][n_seeds][2] final points.
 *   R_out     : float32 [n_events][n_seeds] response at sigma_q.
 *   status    : uint8 [n_events][n_seeds]: 0 ok, 1 some line search took no
 *               step, 2 final point outside the box, 3 non-finite.
 *   n_evals   : nullable uint8 [n_events][n_seeds]: number of R-only passes
 *               over the hits the seed used (its line-search trials); with
 *               the q passes of R, grad R and Hess R this is the seed's exact
 *               work, in units of the paper's T0 (R_out needs no extra pass:
 *               it is the accepted trial's response, or the last pass's R).
 */
int retina_local_search(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events, int32_t model,
                        const float *seeds, int32_t n_seeds, const retina_ls_opts *opts, const retina_grid *box,
                        float *theta_out, float *R_out, uint8_t *status, uint8_t *n_evals, void *stream);

/*
 * retina_refine_maxima - track parameters of each grid cluster, refined from
 * its maximum.
 *
 * Paper: Section 2, step 4 of the grid algorithm (for each selected cluster,
 * estimate the track parameters).  The estimate starts from the cluster's
 * maximum - its cell centre, as retina_grid_scan / retina_grid_maxima write
 * it in max_theta - and takes opts->q truncated-Newton updates of Section 3,
 * exactly the update of retina_local_search (steps 1-4 there), so each
 * point's result is bitwise what retina_local_search gives for the same
 * start, opts and box.  The reading behind the defaults of the bindings:
 * opts->sigma[j] = the grid's own bandwidth for every j, q = 4 updates, each
 * step capped to 1 cell; at that bandwidth the peak is about one cell wide
 * and Newton converges from anywhere inside the cell.  Scheduling is
 * retina_batched_search's (one persistent launch; its RETINA_OPT_BATCH_*
 * options set the launch shape), with each event's points taken from a row
 * of theta_c instead of a ragged array.
 *
 *   theta_c   : float32 [n_events][K][2] starting points (the maxima's cell
 *               centres); only the first min(n_max[e], K) rows of event e are
 *               read (n_max[e] may exceed K, as the grid entry points write
 *               it; negative counts as 0).
 *   n_max     : int32 [n_events], device.
 *   opts, box : host pointers, as in retina_local_search; box is the grid
 *               the maxima come from (step cap in its cells, status 2).
 *   theta_out : float32 [n_events][K][2];  R_out: float32 [n_events][K]
 *               (response at opts->sigma[q-1]);  status: uint8 [n_events][K]
 *               with retina_local_search's codes.  Only the rows that are
 *               read are written; the others keep their contents.  Outputs
 *               must not overlap theta_c.
 *   boxes     : nullable block boxes from retina_prepare_hits (exact
 *               skipping, as in retina_local_search).
 *   ws        : device workspace of retina_refine_maxima_workspace_size bytes
 *               (256-byte aligned), used as retina_batched_search uses its own.
 * Returns RETINA_EINVAL for bad sizes, options or null pointers,
 * RETINA_ENOSPACE for a short workspace (nothing launched in either case);
 * n_events == 0 or K == 0 is a no-op.
 */
int retina_refine_maxima_workspace_size(int32_t n_events, size_t *bytes);
int retina_refine_maxima(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes,
                         int32_t n_events, int32_t model, const float *theta_c, const int32_t *n_max, int32_t K,
                         const retina_ls_opts *opts, const retina_grid *box, float *theta_out, float *R_out,
                         uint8_t *status, void *ws, size_t ws_bytes, void *stream);

/*
 * retina_local_search4 - Algorithm 1 for a four-parameter straight track.
 *
 * Paper: Algorithm 1 with the truncated Newton update of Section 3, for the
 * track theta = (x0, y0, t_x, t_y) at the reference plane z_ref, crossing
 * the layer z at (x0 + t_x w, y0 + t_y w), w = z - z_ref: a line that need
 * not pass through the origin, so a smeared vertex is representable.  s is
 * the in-layer distance of Eq. 1 as for the slope model.  z_ref at the
 * layers' mean z decouples offsets from slopes.  Update j at sigma_j:
 *   1. R, grad R (4) and Hess R (4 x 4) at theta, one pass over the hits.
 *   2. Newton-CG (Nocedal & Wright, Algorithm 7.1) in the variables scaled
 *      by D = diag(scale): CG on (D B D) y = D g, B = -Hess R, from y = 0,
 *      forcing tolerance min(1/2, sqrt|D g|) |D g|, at most 4 iterations;
 *      non-positive curvature: y = D g at the first iteration, else the
 *      current iterate; p = D y.
 *   3. If max_a |p_a| / scale_a > step_cap, p is scaled down to it.
 *   4. Armijo backtracking as in retina_local_search.
 * No block skipping (slope-model boxes do not bound offsets); hits are
 * staged per event in shared memory (RETINA_OPT_LS_SMEM_HITS), the rest read
 * from global memory.
 *
 *   seeds     : float32 [n_events][n_seeds][4] starting points.
 *   seed_count: nullable int32 [n_events]: event e searches its first
 *               min(max(seed_count[e], 0), n_seeds) seeds (the n_seeds of
 *               retina_pair_seeds4 can be passed as is); the outputs of the
 *               others are left untouched.
 *   opts      : host pointer (below).
 *   theta_out : float32 [n_events][n_seeds][4];  R_out: float32
 *               [n_events][n_seeds] at sigma_q;  status: uint8
 *               [n_events][n_seeds]: 0 ok, 1 some line search took no step,
 *               3 non-finite.
 * Returns RETINA_EINVAL for bad sizes, options or null pointers (nothing
 * launched); n_events == 0 or n_seeds == 0 is a no-op.
 */
typedef struct {
    int32_t q;            /* updates per seed, 1 .. RETINA_MAX_Q              */
    float sigma[8];       /* bandwidth at update j                            */
    float c1;             /* Armijo sufficient-increase constant, in [0, 1)  */
    int32_t max_halvings; /* backtracking halvings after t = 1, 0 .. 30      */
    float scale[4];       /* unit of each parameter (CG scaling, step cap), > 0 */
    float step_cap;       /* cap on max_a |p_a| / scale_a, > 0               */
    float zref;           /* reference plane of the offsets (finite)         */
} retina_ls4_opts;
int retina_local_search4(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                         const float *seeds, int32_t n_seeds, const int32_t *seed_count, const retina_ls4_opts *opts,
                         float *theta_out, float *R_out, uint8_t *status, void *stream);

/*
 * retina_pair_seeds4 - starting points for retina_local_search4 from pairs of hits.
 *
 * Paper: none (the paper has no four-parameter search; Algorithm 1 draws its
 * starting points from a prior P_theta it leaves open).  Tracks come from
 * the beam line, so two hits of one track on two layers span a line passing
 * close to the z axis inside the luminous region, while two hits of
 * different tracks rarely do.  For each layer pair p in order
 * (z_a = layer_z[2 p], z_b = layer_z[2 p + 1]), every hit i of the event with
 * |z_i - z_a| <= dz_tol and every hit j with |z_j - z_b| <= dz_tol, in
 * increasing index order (i outer):
 *   t = (x_j - x_i, y_j - y_i) / (z_j - z_i),  |t|^2 = t_x^2 + t_y^2,
 *   kept when |t|^2 > 0, (x_i t_y - y_i t_x)^2 <= d_max^2 |t|^2 (the line's
 *   distance to the z axis is at most d_max) and
 *   zc_lo <= z_i - (x_i t_x + y_i t_y) / |t|^2 <= zc_hi (where it comes
 *   closest);
 *   seed = (x_i + t_x (zref - z_i), y_i + t_y (zref - z_i), t_x, t_y).
 * Every operation is one float32 rounding in the order written (no
 * contraction), so the kept pairs are a function of the float32 inputs.
 *
 *   hits, n_hits, event_offsets, n_events : as retina_local_search4.
 *   layer_z    : host float32 [n_pairs][2], 1 <= n_pairs <= RETINA_MAX_LAYER_PAIRS.
 *   seeds      : float32 [n_events][K][4], the first K kept pairs in order.
 *   n_seeds    : int32 [n_events]: pairs kept (may exceed K), or -1 when a
 *                layer held more than RETINA_PAIR_LAYER_CAP of the event's
 *                hits (then only the first that many of it were paired).
 * Returns RETINA_EINVAL for bad sizes, non-finite or negative cuts or null
 * pointers (nothing launched); n_events == 0 is a no-op.
 */
#define RETINA_MAX_LAYER_PAIRS 8
#define RETINA_PAIR_LAYER_CAP 4096
int retina_pair_seeds4(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                       const float *layer_z, int32_t n_pairs, float dz_tol, float d_max, float zc_lo, float zc_hi,
                       float zref, float *seeds, int32_t *n_seeds, int32_t K, void *stream);

/*
 * retina_batched_search - Algorithm 1 over a ragged batch, one persistent launch.
 *
 * Paper: Algorithm 1 with the Section 3 update, exactly as retina_local_search
 * (same per-seed arithmetic, bitwise the same results for the same seeds),
 * for events of uneven hit and seed counts.  Scheduling: a CTA claims events
 * by an atomic ticket in `order`, stages the event's hits in shared memory
 * and its warps pull groups of seeds from the event's atomic counter; when
 * all events are claimed, CTAs help the events still in progress.  No CTA
 * waits on another; all loops are bounded.
 *
 *   seeds       : float32 [n_seeds][2]; event e owns rows
 *                 seed_offsets[e] .. seed_offsets[e+1]-1 (int64 [n_events+1],
 *                 device; clamped to [0, n_seeds] like the hit offsets).
 *   order       : nullable int32 [n_events] (device): claim order of the events
 *                 (e.g. largest first); entries outside [0, n_events) are
 *                 skipped; NULL means 0, 1, 2, ...  Each event must appear at
 *                 most once.
 *   theta_out, R_out, status, n_evals : per seed, as retina_local_search.
 *   ws, ws_bytes: >= retina_batched_search_workspace_size(n_events) bytes,
 *                 256-byte aligned; zeroed by this call with an async memset on
 *                 `stream` before the kernel (both are stream operations).
 */
int retina_batched_search_workspace_size(int32_t n_events, size_t *bytes);
int retina_batched_search(const float *hits, int64_t n_hits, const int64_t *event_offsets, const float *boxes, int32_t n_events,
                          int32_t model, const float *seeds, int64_t n_seeds, const int64_t *seed_offsets,
                          const int32_t *order, const retina_ls_opts *opts, const retina_grid *box, float *theta_out,
                          float *R_out, uint8_t *status, uint8_t *n_evals, void *ws, size_t ws_bytes, void *stream);

/*
 * retina_sort_seeds - spatial order of each event's starting points.
 *
 * Algorithm 1 treats its starting points independently, so their order is
 * free; consecutive points close in theta need mostly the same hit blocks,
 * which lets retina_batched_search with RETINA_OPT_BATCH_SEEDS_PER_WARP > 1
 * share block tests and hit loads.  Per event (rows seed_offsets[e] ..
 * seed_offsets[e+1]-1, in chunks of 8192): sorted by the Hilbert index
 * (order 9) of the position in `box` quantised to 9 bits per axis (outside
 * points clamp to the edge, non-finite ones go after every finite one), then
 * by original position.  Results of a search on the sorted points belong to
 * the sorted order; perm maps back.
 *
 *   seeds, sorted_out : float32 [n_seeds][2], 8-byte aligned, not the same array.
 *   perm_out  : nullable int32 [n_seeds]: original row of each sorted row.
 */
int retina_sort_seeds(const float *seeds, int64_t n_seeds, const int64_t *seed_offsets, int32_t n_events,
                      const retina_grid *box, float *sorted_out, int32_t *perm_out, void *stream);

/*
 * retina_extract_tracks - cluster the points and keep the best of each.
 *
 * Paper: Algorithm 1, "cluster solutions" and "for each cluster select the
 * solution with the highest response above R0".  Candidates are points with
 * status 0 or 1 (status may be NULL), finite, inside the box and with
 * R >= R0; they are visited by decreasing R (equal R: lower point index
 * first) and a candidate is kept when, for every point kept before it,
 * max_a |theta_a - theta_kept_a| / step_a >= merge_cells.  The comparison is
 * exact (no rounding decides it) when the steps are powers of two.
 *
 *   theta   : float32 [n_events][n_points][2];  R: float32 [n_events][n_points].
 *   status  : nullable uint8 [n_events][n_points].
 *   n_valid : nullable int32 [n_events]; only the first
 *             min(n_valid[e], n_points) points of event e are considered.
 *   tracks  : float32 [n_events][K][2];  track_R: float32 [n_events][K];
 *   track_src: nullable int32 [n_events][K], index of the kept point.
 *   n_tracks: int32 [n_events]; number kept (may exceed K; the first K in
 *             visiting order are written).
 *   n_points must be <= RETINA_MAX_EXTRACT_POINTS (else RETINA_ENOSPACE;
 *   retina_extract_tracks_ws takes more).
 */
int retina_extract_tracks(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                          int32_t n_events, int32_t n_points, const retina_grid *box, float R0,
                          float merge_cells, float *tracks, float *track_R, int32_t *track_src,
                          int32_t *n_tracks, int32_t K, void *stream);

/*
 * retina_extract_tracks_ws - retina_extract_tracks for any number of points.
 *
 * The same rule and outputs as retina_extract_tracks, for n_points up to
 * RETINA_MAX_EXTRACT_POINTS_WS: up to RETINA_MAX_EXTRACT_POINTS points per
 * event the candidates are kept in shared memory as there (ws is not used),
 * beyond that in the caller's workspace, whose size
 * retina_extract_tracks_workspace_size gives (per event one array of keys,
 * coordinates, sources and states for the next power of two >= n_points).
 * Returns RETINA_ENOSPACE (nothing launched) when ws_bytes is too small.
 */
#define RETINA_MAX_EXTRACT_POINTS_WS (1 << 22)
int retina_extract_tracks_workspace_size(int32_t n_events, int32_t n_points, size_t *bytes);
int retina_extract_tracks_ws(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                             int32_t n_events, int32_t n_points, const retina_grid *box, float R0, float merge_cells,
                             float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks, int32_t K,
                             void *ws, size_t ws_bytes, void *stream);

/*
 * retina_extract_tracks4 - cluster / select for four-parameter points.
 *
 * Paper: Algorithm 1, its last two lines, for theta = (x0, y0, t_x, t_y) of
 * retina_local_search4.  Candidates are points with status 0 or 1 (status
 * may be NULL), all four parameters finite, slopes (t_x, t_y) inside
 * slope_box and R >= R0; they are visited by decreasing R (equal R: lower
 * point index first) and a candidate is kept when, for every point kept
 * before it, max_a |theta_a - theta_kept_a| / unit_a >= merge_units.  The
 * comparison is exact when merge_units * unit_a are powers of two.
 *
 *   theta   : float32 [n_events][n_points][4];  R: float32 [n_events][n_points].
 *   n_valid : nullable int32 [n_events]; only the first
 *             min(n_valid[e], n_points) points of event e are considered.
 *   unit    : host float32 [4] > 0 (e.g. the search's scale).
 *   tracks  : float32 [n_events][K][4];  track_R: float32 [n_events][K];
 *   track_src: nullable int32 [n_events][K];  n_tracks: int32 [n_events]
 *             (may exceed K; the first K in visiting order are written).
 *   n_points must be <= RETINA_MAX_EXTRACT_POINTS4 (else RETINA_ENOSPACE).
 */
#define RETINA_MAX_EXTRACT_POINTS4 4096
int retina_extract_tracks4(const float *theta, const float *R, const uint8_t *status, const int32_t *n_valid,
                           int32_t n_events, int32_t n_points, const retina_grid *slope_box, const float *unit, float R0,
                           float merge_units, float *tracks, float *track_R, int32_t *track_src, int32_t *n_tracks,
                           int32_t K, void *stream);

/*
 * Learned seed proposer
 * ---------------------
 * Algorithm 1 starts its local searches from initial guesses drawn from a
 * prior distribution P_theta, which the paper leaves open (a uniform draw
 * over the box is the plain choice).  These entry points replace that prior by
 * a small convolutional network that looks at a coarse histogram of the
 * event's hit slopes and ranks 64 x 64 cells; the K best cells' centres
 * become the seeds.  The proposer is an extension: the paper has no
 * counterpart beyond the prior it replaces.  Only slope-model
 * (RETINA_VELO_SLOPES) hits are supported.
 *
 * Network on one event's 64 x 64 image (row = v bin, column = u bin):
 *   a1 = conv3x3(x; W1, b1) (1 -> 16),  h1 = bf16(relu(a1))
 *   a2 = conv3x3(h1; W2, b2) (16 -> 32), h2 = bf16(relu(a2))
 *   z  = sum_o W3[o] h2[o] + b3          (logits, float32)
 * with 'same' zero padding, stride 1, cross-correlation, every sum in float32
 * and the weights rounded to bfloat16 (round to nearest even) when read.
 * Parameters: float32 [RETINA_SEEDNET_PARAMS] master vector,
 *   W1 [16][1][3][3] at 0, b1 [16] at 144, W2 [32][16][3][3] at 160,
 *   b2 [32] at 4768, W3 [32] at 4800, b3 at 4832.
 * bfloat16 arrays are uint16 bit patterns.
 */
#define RETINA_SEEDNET_BINS 64
#define RETINA_SEEDNET_PARAMS 4833

/*
 * retina_slope_histogram - the network's input image per event.
 *
 * For every hit with |z| >= zmin: u = x / z, v = y / z (float32 division),
 * column floor((u - lo) * s), row floor((v - lo) * s) with s = float32(64 /
 * (hi - lo)), all in float32; hits outside [0, 64) in either bin are dropped.
 * features[e][row][col] = bf16(log1pf(count)).  Counts are exact (integer
 * atomics), so the result does not depend on the hits' order.
 *
 *   hits, n_hits, event_offsets : as everywhere (slope-model rows).
 *   lo < hi finite, zmin >= 0.
 *   features : uint16 (bfloat16) [n_events][64][64].
 *   counts   : nullable int32 [n_events][64][64].
 */
int retina_slope_histogram(const float *hits, int64_t n_hits, const int64_t *event_offsets, int32_t n_events,
                           float lo, float hi, float zmin, uint16_t *features, int32_t *counts, void *stream);

/*
 * retina_seednet_forward - logits of the 64 x 64 cells of each event.
 *
 *   features : uint16 (bfloat16) [n_events][64][64].
 *   params   : float32 [RETINA_SEEDNET_PARAMS].
 *   logits   : float32 [n_events][64][64].
 *   h1       : uint16 (bfloat16) [n_events][16][64][64], required: the first
 *              activation, also the scratch the second layer reads.
 *   h2       : nullable uint16 (bfloat16) [n_events][32][64][64].
 */
int retina_seednet_forward(const uint16_t *features, int32_t n_events, const float *params, float *logits,
                           uint16_t *h1, uint16_t *h2, void *stream);

/*
 * retina_seednet_train_step - one Adam step on binary cross-entropy.
 *
 * Loss over the batch's N = n_events * 4096 pixels (y = labels != 0):
 *   L = (1/N) sum pw y softplus(-z) + (1 - y) softplus(z),
 *   pw = min(100, (N - #pos) / max(#pos, 1)),
 * gradient by back-propagation with dL/da2 and dL/da1 stored as bfloat16 and
 * the weights' bfloat16 rounding passed straight through; every reduction runs
 * in a fixed order, so the step is deterministic.  Then
 * retina_seednet_adam(params, adam_m, adam_v, grad, step, ...).
 *
 *   labels       : uint8 [n_events][64][64].
 *   params, adam_m, adam_v : float32 [RETINA_SEEDNET_PARAMS], updated in place
 *                  (m, v zero before the first step).
 *   step         : Adam step number, >= 1.
 *   loss         : nullable float32 [1]: L at the parameters before the step.
 *   grad         : nullable float32 [RETINA_SEEDNET_PARAMS]: dL/dparams.
 *   ws, ws_bytes : >= retina_seednet_train_workspace_size(n_events), 256-byte
 *                  aligned.
 */
int retina_seednet_train_workspace_size(int32_t n_events, size_t *bytes);
int retina_seednet_train_step(const uint16_t *features, const uint8_t *labels, int32_t n_events, float *params,
                              float *adam_m, float *adam_v, int32_t step, float lr, float beta1, float beta2,
                              float eps, float *loss, float *grad, void *ws, size_t ws_bytes, void *stream);

/*
 * retina_seednet_adam - one Adam update (Kingma & Ba, bias-corrected), float32:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All four arrays float32 [RETINA_SEEDNET_PARAMS]; 0 < b1, b2 < 1; step >= 1.
 */
int retina_seednet_adam(float *params, float *adam_m, float *adam_v, const float *grad, int32_t step, float lr,
                        float beta1, float beta2, float eps, void *stream);

/*
 * retina_topk_seeds - K seeds per event from the ranked cells.
 *
 * Cells are ranked by logit: larger first, equal logits (+0 and -0 alike)
 * by lower cell index (row * 64 + col), NaN below every number.
 * Without hits (hits == NULL): seed j is the centre of the j-th ranked cell,
 *   (lo + (col + 1/2) w, lo + (row + 1/2) w), w = float32((hi - lo) / 64).
 * With the event's hits: the ranked cells are walked in order and each gives
 * seeds until K are out.  A cell splits into 4 x 4 sub-cells (sub-cell of a
 * hit: floor((u - lo) * 4 s) in float32 with the histogram's s and zmin, so
 * it refines the histogram's cell exactly); it gives one seed per sub-cell
 * holding >= min_sub_hits of its hits, fullest first (ties: lower sub-cell
 * row, then column), else one seed for its fullest non-empty sub-cell, else
 * (empty) its centre.  A sub-cell's seed is its hits' mean slope, computed
 * from 2^-32 fixed-point in-sub-cell positions in double and rounded once to
 * float32.  Only the first 1024 ranked cells are split; later cells give
 * their centre.  Two tracks often share a 64 x 64 cell while the local search
 * converges only from a few 1e-3 in slope, hence the split.
 *
 *   logits      : float32 [n_events][64][64], 16-byte aligned (EINVAL otherwise).
 *   K           : 1 .. 4096.
 *   zmin, min_sub_hits (>= 1) : as above; lo, hi as for the histogram.
 *   hits, n_hits, event_offsets : nullable hits (slope-model rows); offsets
 *                 required with hits.
 *   seeds       : float32 [n_events][K][2].
 *   cell_idx    : nullable int32 [n_events][K]: the 64 x 64 cell of each seed.
 */
int retina_topk_seeds(const float *logits, int32_t n_events, int32_t K, float lo, float hi, float zmin,
                      int32_t min_sub_hits, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                      float *seeds, int32_t *cell_idx, void *stream);

/*
 * retina_pipeline_* - one call per batch of events for the whole path.
 *
 * Not a step of the paper: a native executor.  retina_pipeline_run enqueues
 * on the caller's stream the hit ordering (retina_prepare_hits), then, on two
 * concurrent streams, the grid method (retina_grid_response,
 * retina_grid_maxima, retina_extract_tracks of the maxima) and Algorithm 1
 * from the caller's starting points (retina_batched_search and
 * retina_extract_tracks, on a high-priority stream the pipeline owns), and
 * joins both back into the caller's stream.  Results are those of the
 * separate calls with the same launch options.  The pipeline owns its stream,
 * events and device workspace, allocated by retina_pipeline_create for the
 * configured capacities; runs allocate nothing.  Runs of one pipeline must be
 * ordered (one stream, or synchronised): they share the workspace.
 *
 * retina_pipeline_config:
 *   model, grid, sigma_grid, R0 : the grid method (as retina_grid_scan).
 *   opts        : Algorithm 1's options (as retina_batched_search); grid is
 *                 also the search's box.
 *   merge_cells : extraction merge distance in cells (both methods).
 *   max_events, max_hits : capacities of a run.
 *   seeds_per_event : S, every event's number of starting points.
 *   max_maxima  : maxima kept per event by the grid method (K of
 *                 retina_grid_maxima), 1 .. 8192.
 *   max_tracks  : tracks written per event and method (K of
 *                 retina_extract_tracks).
 * retina_pipeline_create validates the configuration before allocating
 * (RETINA_EINVAL, nothing allocated) and returns RETINA_ECUDA when an
 * allocation fails.
 * retina_pipeline_run:
 *   hits, n_hits, event_offsets, n_events : as retina_prepare_hits
 *                 (n_events <= max_events, n_hits <= max_hits).
 *   seeds       : float32 [n_events][S][2].
 *   grid_tracks, grid_track_R, grid_n_tracks : float32 [n_events][max_tracks][2],
 *                 float32 [n_events][max_tracks], int32 [n_events].
 *   search_tracks, search_track_R, search_n_tracks : the same for the search.
 *   Returns RETINA_ENOSPACE (nothing launched) when the grid's hit-slice
 *   partials for the current RETINA_OPT_GRID_SPLITS exceed the workspace.
 */
typedef struct {
    int32_t model;
    retina_grid grid;
    float sigma_grid;
    float R0;
    float merge_cells;
    retina_ls_opts opts;
    int32_t max_events;
    int64_t max_hits;
    int32_t seeds_per_event;
    int32_t max_maxima;
    int32_t max_tracks;
} retina_pipeline_config;

typedef struct retina_pipeline retina_pipeline;

int retina_pipeline_create(const retina_pipeline_config *config, retina_pipeline **out);
int retina_pipeline_run(retina_pipeline *p, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                        int32_t n_events, const float *seeds, float *grid_tracks, float *grid_track_R,
                        int32_t *grid_n_tracks, float *search_tracks, float *search_track_R,
                        int32_t *search_n_tracks, void *stream);
int retina_pipeline_destroy(retina_pipeline *p);

/*
 * retina_tracker_* - Algorithm 1 over a batch of events in one call, replayed
 * as one CUDA graph.
 *
 * Paper: Algorithm 1 (starting points from a prior, the Section 3 updates,
 * cluster / select) over many events; the tracker itself is not a step of
 * the paper but a native executor of the batched search.  A step is: the hit
 * ordering (retina_prepare_hits); the starting points - the learned
 * proposer (retina_slope_histogram over [-0.5, 0.5)^2 with |z| >= 50,
 * retina_seednet_forward, retina_topk_seeds with 3 hits per sub-cell) when
 * the tracker was created with network parameters, else the caller's; their
 * spatial order (retina_sort_seeds) when configured; the persistent batched
 * search (retina_batched_search); cluster / select (retina_extract_tracks).
 * Slope-model (RETINA_VELO_SLOPES) hits only.  The tracker owns its input and
 * output buffers and its workspace, allocated by retina_tracker_create for
 * the configured capacities; steps allocate nothing.  The first step with a
 * given event count and search launch shape records the step's launches in a
 * CUDA graph (when use_graph is set); later steps with the same count and
 * shape replay it.  Steps of one tracker must be ordered (one stream, or
 * synchronised): they share the buffers.
 *
 * retina_tracker_config:
 *   box         : the search box and grid step (step cap, in-box test,
 *                 extraction), as retina_batched_search's box.
 *   opts        : Algorithm 1's options (as retina_batched_search).
 *   R0, merge_cells : extraction (as retina_extract_tracks).
 *   max_events (1 .. 65535), max_hits : capacities of a step.
 *   seeds_per_event : S, every event's starting points (1 .. 8192).
 *   max_tracks  : tracks written per event (K of retina_extract_tracks).
 *   sort_seeds  : 1 = order each event's starting points spatially first.
 *   seeds_per_warp (0, 1, 2, 4), warps (0, 8, 16, 32), smem_hits (0 .. 12288),
 *   ctas        : the batched search's launch shape; 0 = the process-wide
 *                 option (RETINA_OPT_BATCH_*) in force at the step.
 *   use_graph   : 1 = record / replay CUDA graphs, 0 = enqueue the launches.
 * retina_tracker_create(config, seednet_params, &t): seednet_params is NULL
 *   (the caller supplies starting points) or float32 [RETINA_SEEDNET_PARAMS]
 *   in host or device memory, copied at creation.  RETINA_EINVAL (nothing
 *   allocated) for an invalid configuration, RETINA_ECUDA when an allocation
 *   fails.
 * retina_tracker_buffers: device addresses of the owned buffers - hits
 *   float32 [max_hits][4], event_offsets int64 [max_events + 1], seeds
 *   float32 [max_events][S][2] (written by the proposer in learned mode),
 *   tracks float32 [max_events][max_tracks][2], track_R float32
 *   [max_events][max_tracks], n_tracks int32 [max_events] (as
 *   retina_extract_tracks).  Any pointer argument may be NULL.
 * retina_tracker_step(t, n_events, stream): one step on the owned input
 *   buffers (which the caller filled: hits and offsets of n_events events,
 *   offsets[n_events] <= max_hits; seeds unless learned), outputs in the owned
 *   output buffers.
 * retina_tracker_set_marks(t, events, n): n = RETINA_TRACKER_MARKS cudaEvent_t
 *   handles (created by the caller, with timing for durations) that every
 *   later step records - as event nodes of its graph - before the hit
 *   ordering (0), after it (1), after the starting points (2), after their
 *   ordering (3), after the search (4) and after cluster / select (5); n = 0
 *   removes them.  The events stay the caller's; a graph recorded earlier is
 *   recorded again at the next step.
 * retina_tracker_run_host: one step from host memory - copies n_hits hits,
 *   n_events + 1 offsets and (caller seeds only) n_events * S seeds in,
 *   steps, copies n_events rows of tracks, track_R and n_tracks out; the call
 *   returns before the copies finish: synchronise the stream before reading
 *   the host outputs.  Everything but the hit copy is enqueued on `stream` in
 *   that order.  The hit copy runs on the tracker's own copy stream as soon
 *   as the previous step's hit ordering has finished (the only launch that
 *   reads the unsorted hits), so consecutive calls overlap one step's copy
 *   with the previous step's search; the step waits for it.  So the host hit
 *   buffer must hold this step's hits when the call is made (it is not
 *   ordered after work already enqueued on `stream`), and must not change
 *   until `stream` has passed the step.  Host buffers should be page-locked
 *   for the copies to be asynchronous.  The offsets are checked on the host
 *   (non-decreasing, within [0, n_hits]): RETINA_EINVAL, nothing enqueued.
 */
typedef struct {
    retina_grid box;
    retina_ls_opts opts;
    float R0;
    float merge_cells;
    int32_t max_events;
    int64_t max_hits;
    int32_t seeds_per_event;
    int32_t max_tracks;
    int32_t sort_seeds;
    int32_t seeds_per_warp;
    int32_t warps;
    int32_t smem_hits;
    int32_t ctas;
    int32_t use_graph;
} retina_tracker_config;

typedef struct retina_tracker retina_tracker;

#define RETINA_TRACKER_MARKS 6

int retina_tracker_create(const retina_tracker_config *config, const float *seednet_params, retina_tracker **out);
int retina_tracker_buffers(retina_tracker *t, float **hits, int64_t **event_offsets, float **seeds, float **tracks,
                           float **track_R, int32_t **n_tracks);
int retina_tracker_set_marks(retina_tracker *t, void *const *events, int32_t n);
int retina_tracker_step(retina_tracker *t, int32_t n_events, void *stream);
int retina_tracker_run_host(retina_tracker *t, const float *hits, int64_t n_hits, const int64_t *event_offsets,
                            int32_t n_events, const float *seeds, float *tracks, float *track_R, int32_t *n_tracks,
                            void *stream);
int retina_tracker_destroy(retina_tracker *t);

#ifdef __cplusplus
}
#endif

#endif /* RETINA_H */
