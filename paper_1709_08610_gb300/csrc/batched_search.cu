// Algorithm 1 over a ragged batch of events in one persistent launch.
//
// Work is claimed, never waited for:
//  * a CTA claims the next event with an atomic ticket (in the caller's
//    order, e.g. largest first), stages its hits in shared memory once, and
//    its warps pull groups of P seeds from the event's atomic group counter
//    until the event is exhausted;
//  * when every event has been claimed, CTAs help events still in progress
//    (the first with groups left, scanned by the whole CTA), so one large
//    event spreads over the whole GPU and the batch's tail balances.
// No CTA ever waits on another CTA: the only waits are __syncthreads inside a
// CTA, and every loop is bounded by the number of events and seeds.  The
// counters live in the caller's workspace and are zeroed by an async memset
// on the same stream before the launch.
//
// The same kernel refines grid maxima (step 4 of the grid algorithm): the
// starting points are then rows of a [n_events][stride] array with a count
// per event, instead of a ragged array with offsets.
#include "search_device.cuh"

namespace retina {

struct BatchArgs {
    const float4 *hits;
    int64_t n_hits;
    const int64_t *hit_off;
    const float4 *boxes;
    int n_events;
    const float *seeds;
    int64_t n_seeds;
    const int64_t *seed_off;
    const int32_t *order;
    int smem_hits;
    int box_cap;  // block boxes staged per event (a multiple of 4)
    int64_t max_rounds;
    float *theta_out;
    float *R_out;
    uint8_t *status;
    uint8_t *n_evals;
    int32_t *counters;  // [0] event ticket, [1] overrun flag, [2 + e] group counter of event e
    unsigned long long *work;
    const int32_t *seed_count;  // non-null: event e's seeds are e * seed_stride + [0, seed_count[e])
    int64_t seed_stride;
};

__device__ __forceinline__ void seed_range(const BatchArgs &a, int e, int64_t &s0, int64_t &s1) {
    int64_t x, y;
    if (a.seed_count) {
        const int64_t c = a.seed_count[e];
        x = (int64_t)e * a.seed_stride;
        y = x + (c < 0 ? 0 : (c > a.seed_stride ? a.seed_stride : c));
    } else {
        x = a.seed_off[e];
        y = a.seed_off[e + 1];
    }
    x = x < 0 ? 0 : (x > a.n_seeds ? a.n_seeds : x);
    y = y < x ? x : (y > a.n_seeds ? a.n_seeds : y);
    s0 = x;
    s1 = y;
}

template <int P>
__device__ __forceinline__ int64_t n_groups_of(const BatchArgs &a, int e) {
    int64_t s0, s1;
    seed_range(a, e, s0, s1);
    return (s1 - s0 + P - 1) / P;
}

template <int MODEL, int P>
__host__ __device__ constexpr bool batch_smem_state() { return P == 4 && MODEL == RETINA_VELO_SLOPES; }

template <int MODEL, int P>
constexpr size_t batch_state_bytes(int warps) {
    return batch_smem_state<MODEL, P>() ? (size_t)warps * ((sizeof(GroupState<P>) + 15) / 16 * 16) : 0;
}

// at most 64 registers per thread: 2048 / (32 WARPS) CTAs of WARPS warps fit the register file
template <int MODEL, int P, int WARPS, int UPD, bool RL>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) batched_search_kernel(BatchArgs a, LsParams prm) {
    extern __shared__ float4 sh[];
    __shared__ int cur_e;
    pdl_release();  // the track extraction may be scheduled once every CTA has started
    const int tid = threadIdx.x, lane = tid & 31;
    float4 *sbox = staged_box_bounds(sh, a.smem_hits);
    float *sz2 = staged_box_z2(sh, a.smem_hits, a.box_cap);
    float4 *ssb = staged_super_bounds(sh, a.smem_hits, a.box_cap);
    float *ssz2 = staged_super_z2(sh, a.smem_hits, a.box_cap);
    int *list = kept_list(sh, a.smem_hits, a.box_cap, tid >> 5);
    // four seeds per warp keep their warp-uniform state in shared memory, one
    // copy per warp after the lists (see batch_state_bytes)
    constexpr bool SS = batch_smem_state<MODEL, P>();
    GroupState<P> *gstate = nullptr;
    if constexpr (SS)
        gstate = reinterpret_cast<GroupState<P> *>(reinterpret_cast<unsigned char *>(sh) +
                                                   search_smem_bytes(a.smem_hits, a.boxes != nullptr, WARPS,
                                                                     a.box_cap)) + (tid >> 5);
    int staged = -1;
    int n_staged = 0, n_sbox = 0;
    for (int64_t round = 0; round < a.max_rounds; ++round) {
        // ---- pick an event: the next unclaimed one, else one still in progress
        if (tid == 0) {
            const int c = atomicAdd(&a.counters[0], 1);
            int e = -1;
            if (c < a.n_events) {
                e = a.order ? a.order[c] : c;
                if (e < 0 || e >= a.n_events) e = -2;  // invalid order entry: nothing to do this round
            }
            cur_e = e;
        }
        __syncthreads();
        int e = cur_e;
        __syncthreads();  // every thread has read cur_e before it is written again
        if (e == -1) {
            // all claimed: help the first event (from a CTA-dependent start) with groups left
            if (tid == 0) cur_e = 0x7fffffff;
            __syncthreads();
            for (int i = tid; i < a.n_events; i += blockDim.x) {
                const int ev = (int)((i + (int64_t)blockIdx.x * 7) % a.n_events);
                const int64_t taken = *((volatile int32_t *)&a.counters[2 + ev]);
                if (taken < n_groups_of<P>(a, ev)) atomicMin(&cur_e, ev);
            }
            __syncthreads();
            e = cur_e;
            __syncthreads();
            if (e == 0x7fffffff) break;  // every event is exhausted
        }
        if (e < 0) continue;
        int64_t hb, he, s0, s1;
        event_range(a.hit_off, a.n_hits, e, hb, he);
        seed_range(a, e, s0, s1);
        const int H = (int)(he - hb);
        const float4 *gh = a.hits + hb;
        const float4 *gbox = a.boxes ? a.boxes + 2 * (hb / 32 + e) : nullptr;
        if (e != staged) {
            n_staged = H < a.smem_hits ? H : a.smem_hits;
            for (int k = tid; k < n_staged; k += blockDim.x) sh[k] = __ldg(gh + k);
            const int nblk = (H + 31) >> 5, cap = a.box_cap;
            n_sbox = gbox ? (nblk < cap ? nblk : cap) : 0;
            stage_boxes<MODEL>(gbox, n_sbox, sbox, sz2, ssb, ssz2, tid, blockDim.x);
            staged = e;
        }
        __syncthreads();
        const int64_t groups = (s1 - s0 + P - 1) / P;
        for (int64_t it = 0; it <= groups; ++it) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&a.counters[2 + e], 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= groups) break;
            const int64_t s = s0 + (int64_t)g * P;
            const int n_live = (int)((s1 - s) < P ? (s1 - s) : P);
            search_group<MODEL, P, UPD, SS, RL>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list,
                                            a.seeds + 2 * s, n_live, prm, a.theta_out + 2 * s, a.R_out + s,
                                            a.status + s, a.n_evals ? a.n_evals + s : nullptr, a.work, gstate);
        }
        __syncthreads();  // all warps done with the staged hits before the next round
        if (round + 1 == a.max_rounds && tid == 0) atomicExch(&a.counters[1], 1);
    }
}

size_t batched_ws_bytes(int n_events) { return ((size_t)(n_events + 2) * sizeof(int32_t) + 255) / 256 * 256; }

template <int MODEL, int P, int WARPS, int UPD, bool RL = false>
static cudaError_t launch_batched_t(BatchArgs a, const LsParams &prm, int ctas, cudaStream_t st) {
    auto kern = batched_search_kernel<MODEL, P, WARPS, UPD, RL>;
    // boxes take the shared memory the hits and the warps' lists leave (at
    // least the staged hits' blocks, at most 4096 blocks = 131072 hits)
    a.box_cap = default_box_cap(a.smem_hits);
    if (a.boxes) {
        const size_t avail = (size_t)max_dynamic_smem() - 1024;  // static shared memory and a margin
        const size_t fixed = (size_t)a.smem_hits * 16 + search_list_bytes(WARPS) + batch_state_bytes<MODEL, P>(WARPS);
        if (avail > fixed) {
            int cap = (int)((avail - fixed) / 25) & ~3;  // 20 B per block box + 5 B of its superblock's
            cap = cap > 4096 ? 4096 : cap;
            if (cap > a.box_cap) a.box_cap = cap;
        }
    }
    const size_t smem =
        search_smem_bytes(a.smem_hits, a.boxes != nullptr, WARPS, a.box_cap) + batch_state_bytes<MODEL, P>(WARPS);
    cudaError_t aerr = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (aerr != cudaSuccess) return aerr;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    // persistent: as many CTAs as fit at once, or fewer when the caller leaves room for concurrent kernels
    const int fill = per_sm * sm_count();
    const int grid = (ctas > 0 && ctas < fill) ? ctas : fill;
    // latency-bound (at most two seed groups per resident warp): pair the trials
    LsParams p2 = prm;
    p2.pair_trials = (a.n_seeds + P - 1) / P <= 2LL * grid * WARPS ? 1 : 0;
    PrioLaunch L(dim3(grid), dim3(WARPS * 32), smem, st);
    const cudaError_t lerr = cudaLaunchKernelEx(&L.cfg, kern, a, p2);
    count_launches(1);
    return lerr != cudaSuccess ? lerr : cudaGetLastError();
}

template <int MODEL, int P, int UPD = RETINA_UPDATE_TRUNCATED_NEWTON>
static cudaError_t launch_batched_w(int warps, const BatchArgs &a, const LsParams &prm, int ctas, cudaStream_t st) {
    // four packed slope-model seeds on events of at most 128 blocks on
    // average: the kernel whose updates keep one kept-block list for their
    // trials (a separate instantiation, so the other shapes' code is untouched)
    if constexpr (MODEL == RETINA_VELO_SLOPES && P == 4 && UPD == RETINA_UPDATE_TRUNCATED_NEWTON) {
        if (a.boxes && a.n_hits <= (int64_t)a.n_events * 32 * KEPT_CHUNK) {
            if (warps >= 32) return launch_batched_t<MODEL, P, 32, UPD, true>(a, prm, ctas, st);
            if (warps >= 16) return launch_batched_t<MODEL, P, 16, UPD, true>(a, prm, ctas, st);
            return launch_batched_t<MODEL, P, 8, UPD, true>(a, prm, ctas, st);
        }
    }
    if (warps >= 32) return launch_batched_t<MODEL, P, 32, UPD>(a, prm, ctas, st);
    if (warps >= 16) return launch_batched_t<MODEL, P, 16, UPD>(a, prm, ctas, st);
    return launch_batched_t<MODEL, P, 8, UPD>(a, prm, ctas, st);
}

static cudaError_t launch_batched(BatchArgs &a, int model, const retina_ls_opts *o, const retina_grid *box,
                                  int seeds_per_warp, int warps, int ctas, cudaStream_t st) {
    LsParams prm = make_ls_params(o, box);
    if (a.smem_hits < 0) a.smem_hits = 0;
    if (a.smem_hits > 12288) a.smem_hits = 12288;
    a.max_rounds = (int64_t)a.n_events + a.n_seeds + 2;
    a.work = work_counters();
    cudaError_t err = cudaMemsetAsync(a.counters, 0, batched_ws_bytes(a.n_events), st);
    if (err != cudaSuccess) return err;
    // the comparison updates run one seed per warp (bitwise the same results
    // as any other grouping), which keeps their instantiations few
    if (o->update == RETINA_UPDATE_STEEPEST_ASCENT)
        return model == RETINA_VELO_SLOPES
                   ? launch_batched_w<RETINA_VELO_SLOPES, 1, RETINA_UPDATE_STEEPEST_ASCENT>(warps, a, prm, ctas, st)
                   : launch_batched_w<RETINA_TOY2D, 1, RETINA_UPDATE_STEEPEST_ASCENT>(warps, a, prm, ctas, st);
    if (o->update == RETINA_UPDATE_MODIFIED_NEWTON)
        return model == RETINA_VELO_SLOPES
                   ? launch_batched_w<RETINA_VELO_SLOPES, 1, RETINA_UPDATE_MODIFIED_NEWTON>(warps, a, prm, ctas, st)
                   : launch_batched_w<RETINA_TOY2D, 1, RETINA_UPDATE_MODIFIED_NEWTON>(warps, a, prm, ctas, st);
#define RETINA_BATCH_CASE(M, PP) return launch_batched_w<M, PP>(warps, a, prm, ctas, st)
    if (model == RETINA_VELO_SLOPES) {
        if (seeds_per_warp >= 4) RETINA_BATCH_CASE(RETINA_VELO_SLOPES, 4);
        if (seeds_per_warp == 2) RETINA_BATCH_CASE(RETINA_VELO_SLOPES, 2);
        RETINA_BATCH_CASE(RETINA_VELO_SLOPES, 1);
    } else {
        if (seeds_per_warp >= 4) RETINA_BATCH_CASE(RETINA_TOY2D, 4);
        if (seeds_per_warp == 2) RETINA_BATCH_CASE(RETINA_TOY2D, 2);
        RETINA_BATCH_CASE(RETINA_TOY2D, 1);
    }
#undef RETINA_BATCH_CASE
}

cudaError_t launch_batched_search(const float4 *hits, int64_t n_hits, const int64_t *hit_off, const float4 *boxes,
                                  int n_events, int model,
                                  const float *seeds, int64_t n_seeds, const int64_t *seed_off, const int32_t *order,
                                  const retina_ls_opts *o, const retina_grid *box, float *theta_out, float *R_out,
                                  uint8_t *status, uint8_t *n_evals, int32_t *counters, int seeds_per_warp, int warps,
                                  int smem_hits, int ctas, cudaStream_t st) {
    BatchArgs a{hits, n_hits, hit_off, boxes, n_events, seeds, n_seeds, seed_off, order, smem_hits, 0, 0,
                theta_out, R_out, status, n_evals, counters, nullptr, nullptr, 0};
    return launch_batched(a, model, o, box, seeds_per_warp, warps, ctas, st);
}

cudaError_t launch_refine_maxima(const float4 *hits, int64_t n_hits, const int64_t *hit_off, const float4 *boxes,
                                 int n_events, int model, const float *theta_c, const int32_t *n_max, int K,
                                 const retina_ls_opts *o, const retina_grid *box, float *theta_out, float *R_out,
                                 uint8_t *status, int32_t *counters, int seeds_per_warp, int warps, int smem_hits,
                                 int ctas, cudaStream_t st) {
    BatchArgs a{hits, n_hits, hit_off, boxes, n_events, theta_c, (int64_t)n_events * K, nullptr, nullptr, smem_hits,
                0, 0, theta_out, R_out, status, nullptr, counters, nullptr, n_max, (int64_t)K};
    return launch_batched(a, model, o, box, seeds_per_warp, warps, ctas, st);
}

}  // namespace retina
