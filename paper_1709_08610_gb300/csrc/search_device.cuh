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
        // every operation rounded explicitly (no contraction), so that the
        // packed two-seed form (RghAcc2) gives bitwise the same sums
        const float rx = __fmaf_rn(-t0, h.z, h.x);
        const float ry = __fmaf_rn(-t1, h.z, h.y);
        const float s2 = __fmaf_rn(rx, rx, __fmul_rn(ry, ry));
        const float e = ex2_mufu(__fmul_rn(s2, -kk));
        const float ez = __fmul_rn(e, h.z);
        const float ez2 = __fmul_rn(ez, h.z);
        const float ez2rx = __fmul_rn(ez2, rx);
        S[0] = __fadd_rn(S[0], e);
        S[1] = __fmaf_rn(ez, rx, S[1]);
        S[2] = __fmaf_rn(ez, ry, S[2]);
        S[3] = __fmaf_rn(ez2rx, rx, S[3]);
        S[4] = __fmaf_rn(ez2rx, ry, S[4]);
        S[5] = __fmaf_rn(__fmul_rn(ez2, ry), ry, S[5]);
        S[6] = __fadd_rn(S[6], ez2);
    } else {
        const float r = __fsub_rn(__fmaf_rn(-t0, h.x, h.y), t1);
        const float e = ex2_mufu(__fmul_rn(__fmul_rn(r, r), -kk));
        const float er = __fmul_rn(e, r);
        const float erx = __fmul_rn(er, h.x);
        const float ex = __fmul_rn(e, h.x);
        S[0] = __fadd_rn(S[0], e);
        S[1] = __fadd_rn(S[1], erx);
        S[2] = __fadd_rn(S[2], er);
        S[3] = __fmaf_rn(__fmul_rn(erx, r), h.x, S[3]);
        S[4] = __fmaf_rn(erx, r, S[4]);
        S[5] = __fmaf_rn(er, r, S[5]);
        S[6] = __fmaf_rn(ex, h.x, S[6]);
        S[7] = __fadd_rn(S[7], ex);
    }
}

template <int MODEL>
__device__ __forceinline__ float pair_r(const float4 h, float t0, float t1, float kk) {
    if (MODEL == RETINA_VELO_SLOPES) {
        const float rx = __fmaf_rn(-t0, h.z, h.x);
        const float ry = __fmaf_rn(-t1, h.z, h.y);
        return ex2_mufu(__fmul_rn(__fmaf_rn(rx, rx, __fmul_rn(ry, ry)), -kk));
    } else {
        const float r = __fsub_rn(__fmaf_rn(-t0, h.x, h.y), t1);
        return ex2_mufu(__fmul_rn(__fmul_rn(r, r), -kk));
    }
}

// Accumulators of the RGH sums of one point (add2: hit a, then hit b).
// Packing the pair arithmetic into FP32x2 instructions was measured slower
// here (register pressure and operand moves outweighed the saved issue
// slots), so the sums use the scalar pair_rgh.
template <int MODEL>
struct RghAcc {
    float S[Model<MODEL>::NS];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < Model<MODEL>::NS; ++i) S[i] = 0.f;
    }
    __device__ __forceinline__ void add(const float4 h, float t0, float t1, float kk) {
        pair_rgh<MODEL>(h, t0, t1, kk, S);
    }
    __device__ __forceinline__ void add2(const float4 a, const float4 b, float t0, float t1, float kk) {
        pair_rgh<MODEL>(a, t0, t1, kk, S);
        pair_rgh<MODEL>(b, t0, t1, kk, S);
    }
    __device__ __forceinline__ void sums(float *out) const {
#pragma unroll
        for (int i = 0; i < Model<MODEL>::NS; ++i) out[i] = S[i];
    }
};

// R-only terms of two hits, added to Rt in the order a, b.
template <int MODEL>
__device__ __forceinline__ void pair_r2(const float4 a, const float4 b, float t0, float t1, float kk, float &Rt) {
    Rt = __fadd_rn(Rt, pair_r<MODEL>(a, t0, t1, kk));
    Rt = __fadd_rn(Rt, pair_r<MODEL>(b, t0, t1, kk));
}

// The RGH sums of two points (seeds a and b of a warp) over the same hits, in
// packed FP32x2 arithmetic: lane lo is seed a, hi is seed b, and each packed
// operation rounds every lane exactly as the scalar operation of pair_rgh
// does, so the sums are bitwise RghAcc's (slope model only).  One packed
// instruction does the work of two scalar ones; the hit's coordinates are
// broadcast into both lanes.
struct RghAcc2 {
    unsigned long long S[7];
    unsigned long long nt0, nt1, nkk;  // (-t0a, -t0b), (-t1a, -t1b), (-kk, -kk)
    __device__ __forceinline__ void set(float t0a, float t1a, float t0b, float t1b, float kk) {
        nt0 = pack2(-t0a, -t0b);
        nt1 = pack2(-t1a, -t1b);
        nkk = pack2(-kk, -kk);
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 7; ++i) S[i] = 0ull;
    }
    __device__ __forceinline__ void add(const float4 h) {
        const unsigned long long X = pack2(h.x, h.x), Y = pack2(h.y, h.y), Z = pack2(h.z, h.z);
        const unsigned long long rx = fma2_rn(nt0, Z, X);
        const unsigned long long ry = fma2_rn(nt1, Z, Y);
        const unsigned long long s2 = fma2_rn(rx, rx, mul2_rn(ry, ry));
        float a0, a1;
        unpack2(mul2_rn(s2, nkk), a0, a1);
        const unsigned long long e = pack2(ex2_mufu(a0), ex2_mufu(a1));
        const unsigned long long ez = mul2_rn(e, Z);
        const unsigned long long ez2 = mul2_rn(ez, Z);
        const unsigned long long ez2rx = mul2_rn(ez2, rx);
        S[0] = add2_rn(S[0], e);
        S[1] = fma2_rn(ez, rx, S[1]);
        S[2] = fma2_rn(ez, ry, S[2]);
        S[3] = fma2_rn(ez2rx, rx, S[3]);
        S[4] = fma2_rn(ez2rx, ry, S[4]);
        S[5] = fma2_rn(mul2_rn(ez2, ry), ry, S[5]);
        S[6] = add2_rn(S[6], ez2);
    }
    __device__ __forceinline__ void sums(float *a, float *b) const {
#pragma unroll
        for (int i = 0; i < 7; ++i) unpack2(S[i], a[i], b[i]);
    }
};

// R-only terms of one hit for two points in packed form, added to the packed
// Rt (lo: point a, hi: point b); bitwise pair_r + __fadd_rn per lane.
__device__ __forceinline__ void pair_r_x2(const float4 h, unsigned long long nt0, unsigned long long nt1,
                                          unsigned long long nkk, unsigned long long &Rt) {
    const unsigned long long X = pack2(h.x, h.x), Y = pack2(h.y, h.y), Z = pack2(h.z, h.z);
    const unsigned long long rx = fma2_rn(nt0, Z, X);
    const unsigned long long ry = fma2_rn(nt1, Z, Y);
    float a0, a1;
    unpack2(mul2_rn(fma2_rn(rx, rx, mul2_rn(ry, ry)), nkk), a0, a1);
    Rt = add2_rn(Rt, pack2(ex2_mufu(a0), ex2_mufu(a1)));
}

template <int MODEL>
__device__ __forceinline__ void sums_to_rgh(const float *S, float k, float &R, float &g0, float &g1, float &H00,
                                            float &H01, float &H11) {
    // every operation rounded explicitly, so that each search shape (one
    // point per warp, groups, lane-parallel epilogues) computes the same bits
    const float k2 = __fmul_rn(2.f, k), k4 = __fmul_rn(__fmul_rn(4.f, k), k);
    R = S[0];
    g0 = __fmul_rn(k2, S[1]);
    g1 = __fmul_rn(k2, S[2]);
    if (MODEL == RETINA_VELO_SLOPES) {
        H00 = __fsub_rn(__fmul_rn(k4, S[3]), __fmul_rn(k2, S[6]));
        H01 = __fmul_rn(k4, S[4]);
        H11 = __fsub_rn(__fmul_rn(k4, S[5]), __fmul_rn(k2, S[6]));
    } else {
        H00 = __fsub_rn(__fmul_rn(k4, S[3]), __fmul_rn(k2, S[6]));
        H01 = __fsub_rn(__fmul_rn(k4, S[4]), __fmul_rn(k2, S[7]));
        H11 = __fsub_rn(__fmul_rn(k4, S[5]), __fmul_rn(k2, S[0]));
    }
}

// Directional derivative g . p and the Armijo bound R + c1 t (g . p) of the
// backtracking line search (Algorithm 1), rounded explicitly.
__device__ __forceinline__ float dir_slope(float g0, float g1, float p0, float p1) {
    return __fmaf_rn(g0, p0, __fmul_rn(g1, p1));
}
__device__ __forceinline__ float armijo_bound(float R, float c1, float t, float slope) {
    return __fmaf_rn(__fmul_rn(c1, t), slope, R);
}

// Step cap: scale (p0, p1) so that it moves at most cap grid cells on either axis.
__device__ __forceinline__ void cap_step(float &p0, float &p1, float step0, float step1, float cap) {
    const float cells = fmaxf(__fdiv_rn(fabsf(p0), step0), __fdiv_rn(fabsf(p1), step1));
    if (cells > cap) {
        const float sc = __fdiv_rn(cap, cells);
        p0 = __fmul_rn(p0, sc);
        p1 = __fmul_rn(p1, sc);
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

// Newton direction with a modified Hessian (Nocedal & Wright, Section 3.4):
// B = -H shifted by tau I, tau = max(0, delta - mu1), mu1 <= mu2 the
// eigenvalues of B, delta = 1e-3 max(|mu1|, |mu2|); p solves
// (B + tau I) p = g, or p = g when B = 0.  B and g are scaled by the same
// power of two (B's largest entry into [1/2, 1)), which leaves p unchanged
// and keeps the squares of the eigenvalue formula in range.
__device__ __forceinline__ void modified_newton(float g0, float g1, float H00, float H01, float H11, float &p0,
                                                float &p1) {
    const float m = fmaxf(fmaxf(fabsf(H00), fabsf(H11)), fabsf(H01));
    if (!(m > 0.f) || !isfinite(m)) {
        p0 = g0;
        p1 = g1;
        return;
    }
    int ex;
    frexpf(m, &ex);
    const float c = ldexpf(1.f, -ex);
    const float a = -H00 * c, b = -H01 * c, d = -H11 * c;
    const float mid = 0.5f * (a + d), rad = sqrtf(0.25f * (a - d) * (a - d) + b * b);
    const float mu1 = mid - rad, mu2 = mid + rad;
    const float delta = 1e-3f * fmaxf(fabsf(mu1), fabsf(mu2));
    const float tau = mu1 < delta ? delta - mu1 : 0.f;
    const float a2 = a + tau, d2 = d + tau;
    const float det = a2 * d2 - b * b;
    const float sg0 = g0 * c, sg1 = g1 * c;
    p0 = (d2 * sg0 - b * sg1) / det;
    p1 = (a2 * sg1 - b * sg0) / det;
}

// The direction of one update (RETINA_UPDATE_*), chosen at compile time so
// that the truncated Newton search compiles exactly as without the others.
template <int UPD>
__device__ __forceinline__ void update_direction(float g0, float g1, float H00, float H01, float H11, float &p0,
                                                 float &p1) {
    if constexpr (UPD == RETINA_UPDATE_STEEPEST_ASCENT) {
        p0 = g0;
        p1 = g1;
    } else if constexpr (UPD == RETINA_UPDATE_MODIFIED_NEWTON) {
        modified_newton(g0, g1, H00, H01, H11, p0, p1);
    } else {
        newton_cg(g0, g1, H00, H01, H11, p0, p1);
    }
}

struct LsParams {
    int q;
    float kk[RETINA_MAX_Q];  // log2(e) / sigma_j^2
    float k[RETINA_MAX_Q];   // 1 / sigma_j^2
    float cull[RETINA_MAX_Q];  // CULL_EXPONENT / kk[j]: skipping threshold on |z|min^2 dist^2
    float c1;
    int max_halvings;
    float cap;
    GridDev box;
    // one-seed search: test the backtracking trials t and t/2 in one pass
    // once t = 1 is rejected (the same results in fewer dependent passes,
    // at the cost of the second point's terms when t is accepted); set by
    // the launchers when the launch is latency-bound (few seeds per warp)
    int pair_trials;
};

LsParams make_ls_params(const retina_ls_opts *o, const retina_grid *box);

// Shared-memory layout of the search kernels: smem_hits hits, then (with
// boxes) the boxes of the first box_cap blocks (a multiple of 4) in
// search_box form as two arrays (the slope bounds, float4, then the
// |z|min^2 terms; lanes reading consecutive blocks touch consecutive words),
// the same two arrays for their box_cap / 4 superblocks (the union of 4
// consecutive blocks' boxes), then per warp one list of KEPT_CHUNK
// kept-block offsets and 32 superblock slots.  default_box_cap covers the
// staged hits' blocks; the batched kernel gives the boxes whatever shared
// memory the hits and lists leave (box tests of unstaged blocks cost more
// issue slots than loads of unstaged hits).
constexpr int KEPT_CHUNK = 128;  // blocks tested per chunk of a pass (4 per lane, or 1 superblock per lane)
__host__ __device__ __forceinline__ int default_box_cap(int smem_hits) { return ((smem_hits + 31) / 32 + 1 + 3) & ~3; }
__host__ __device__ __forceinline__ size_t search_list_bytes(int warps) {
    return (size_t)warps * (KEPT_CHUNK + 32) * sizeof(int);
}
__host__ __device__ __forceinline__ size_t search_smem_bytes(int smem_hits, bool with_boxes, int warps, int box_cap) {
    return (size_t)smem_hits * 16 +
           (with_boxes ? (size_t)box_cap * 20 + (size_t)(box_cap / 4) * 20 + search_list_bytes(warps) : 0);
}
__device__ __forceinline__ float4 *staged_box_bounds(float4 *sh, int smem_hits) { return sh + smem_hits; }
__device__ __forceinline__ float *staged_box_z2(float4 *sh, int smem_hits, int box_cap) {
    return reinterpret_cast<float *>(sh + smem_hits + box_cap);
}
__device__ __forceinline__ float4 *staged_super_bounds(float4 *sh, int smem_hits, int box_cap) {
    return reinterpret_cast<float4 *>(staged_box_z2(sh, smem_hits, box_cap) + box_cap);
}
__device__ __forceinline__ float *staged_super_z2(float4 *sh, int smem_hits, int box_cap) {
    return reinterpret_cast<float *>(staged_super_bounds(sh, smem_hits, box_cap) + box_cap / 4);
}
__device__ __forceinline__ int *kept_list(float4 *sh, int smem_hits, int box_cap, int warp) {
    return reinterpret_cast<int *>(staged_super_z2(sh, smem_hits, box_cap) + box_cap / 4) + warp * (KEPT_CHUNK + 32);
}

// Lane-strided pass over an event's hits: the staged prefix from shared
// memory (two hits per iteration for independent work), then the rest, if
// any, straight from global memory through L1.
template <typename F, typename F2>
__device__ __forceinline__ void for_each_hit(const float4 *__restrict__ sh, const float4 *__restrict__ gh,
                                             int n_staged, int H, int lane, F &&f, F2 &&f2) {
    int k = lane;
    for (; k + 32 < n_staged; k += 64) f2(sh[k], sh[k + 32]);
    for (; k < n_staged; k += 32) f(sh[k]);
    for (; k < H; k += 32) f(__ldg(gh + k));
}

// Exact skipping of hit blocks (boxes from retina_prepare_hits).  A block
// can be skipped for a point theta when a lower bound of s^2 * log2(e) /
// sigma^2 over the block's box exceeds CULL_EXPONENT: then every hit of the
// block has ex2(-x) with x > 126, which ex2.approx.ftz returns as exactly
// zero, so its terms add nothing to any sum.  140 leaves a margin over 126
// that covers every relative rounding of the bound (a few float32 ulps).
constexpr float CULL_EXPONENT = 140.f;

// A block box as the search tests it, made once when the box is staged.
// Slope model, box (umin, umax, vmin, vmax | |z|min, ...): the slope
// intervals are widened by S = 1e-6 max|bound|, sixteen times the float32
// rounding of x / z when the box was built, so every hit's exact slope lies
// inside; the returned weight is |z|min^2.  A box with a non-finite value
// becomes the whole plane with weight 0, which the test never skips.  2D toy:
// A unchanged, weight = B.x (0, or -inf for a non-finite box).
template <int MODEL>
__device__ __forceinline__ float search_box(float4 &A, const float4 B) {
    if (MODEL == RETINA_VELO_SLOPES) {
        const bool fin = isfinite(A.x) && isfinite(A.y) && isfinite(A.z) && isfinite(A.w) && isfinite(B.x);
        const float S = 1e-6f * fmaxf(fmaxf(fabsf(A.x), fabsf(A.y)), fmaxf(fabsf(A.z), fabsf(A.w)));
        A = fin ? make_float4(A.x - S, A.y + S, A.z - S, A.w + S) : make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
        return fin ? B.x * B.x : 0.f;
    }
    return B.x;
}

// Stage the boxes of blocks [0, n_sbox) of an event in search_box form and,
// for the slope model, the boxes of their superblocks (4 consecutive blocks;
// the last may hold fewer): the union of the slope bounds and the smallest
// |z|min^2.  A superblock box contains each of its blocks' boxes, so its
// lower bound on the exponent is at most theirs: skipping the superblock
// skips only blocks the per-block test skips.  All threads of the CTA call
// it (thread tid of nthreads); the caller synchronises.
template <int MODEL>
__device__ __forceinline__ void stage_boxes(const float4 *__restrict__ gbox, int n_sbox, float4 *sbox, float *sz2,
                                            float4 *ssb, float *ssz2, int tid, int nthreads) {
    if (MODEL != RETINA_VELO_SLOPES) {
        for (int k = tid; k < n_sbox; k += nthreads) {
            float4 A = __ldg(gbox + 2 * k);
            sz2[k] = search_box<MODEL>(A, __ldg(gbox + 2 * k + 1));
            sbox[k] = A;
        }
        return;
    }
    const int n_super = (n_sbox + 3) >> 2;
    for (int q = tid; q < n_super; q += nthreads) {
        float4 U = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
        float w = INFINITY;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 4 * q + j;
            if (k < n_sbox) {
                float4 A = __ldg(gbox + 2 * k);
                const float z2 = search_box<MODEL>(A, __ldg(gbox + 2 * k + 1));
                sz2[k] = z2;
                sbox[k] = A;
                U = make_float4(fminf(U.x, A.x), fmaxf(U.y, A.y), fminf(U.z, A.z), fmaxf(U.w, A.w));
                w = fminf(w, z2);
            }
        }
        ssb[q] = U;
        ssz2[q] = w;
    }
}

// One point's constants for the skipping test of one pass.  Slope model:
// c = CULL_EXPONENT / kk, the threshold on dist^2 |z|min^2 (infinite, never
// skip, around a non-finite point, whose full sums may be NaN).  2D toy: c = kk.
struct CullPt {
    float t0, t1, c;
};
template <int MODEL>
__device__ __forceinline__ CullPt cull_pt(float t0, float t1, float kk, float cull) {
    if (MODEL == RETINA_VELO_SLOPES) return CullPt{t0, t1, (isfinite(t0) && isfinite(t1)) ? cull : INFINITY};
    return CullPt{t0, t1, kk};
}

// Constants for skipping a block only when it is skippable at both of two
// bandwidths (a pass that sums at both).
template <int MODEL>
__device__ __forceinline__ CullPt cull_pt_union(float t0, float t1, float kk_a, float cull_a, float kk_b,
                                                float cull_b) {
    if (MODEL == RETINA_VELO_SLOPES)
        return CullPt{t0, t1, (isfinite(t0) && isfinite(t1)) ? fmaxf(cull_a, cull_b) : INFINITY};
    return CullPt{t0, t1, fminf(kk_a, kk_b)};
}

// True when every hit of the block (box in search_box form) has
// s^2 log2(e) / sigma^2 > CULL_EXPONENT at the point.  Slope model:
// s^2 = z^2 |(u, v) - theta|^2 >= |z|min^2 dist^2, each distance with one
// rounding (relative).  2D toy, box (xmin, xmax, ymin, ymax): r = y - t0 x - t1
// over the box by interval arithmetic, less a slack of 1e-6 per magnitude
// for the rounding of the bound itself.
template <int MODEL>
__device__ __forceinline__ bool box_culled(const float4 A, const float w, const CullPt &p) {
    if (MODEL == RETINA_VELO_SLOPES) {
        const float du = fmaxf(fmaxf(A.x - p.t0, p.t0 - A.y), 0.f);
        const float dv = fmaxf(fmaxf(A.z - p.t1, p.t1 - A.w), 0.f);
        return __fmaf_rn(du, du, dv * dv) * w > p.c;
    } else {
        if (!isfinite(w)) return false;  // boxes with non-finite hits are infinite
        const float a = p.t0 * A.x, b = p.t0 * A.y;
        const float lo = A.z - p.t1 - fmaxf(a, b), hi = A.w - p.t1 - fminf(a, b);
        const float d = fmaxf(fmaxf(lo, -hi), 0.f);
        const float dd = fmaxf(d - 1e-6f * (fabsf(A.z) + fabsf(A.w) + 2.f * fabsf(p.t1) + fabsf(a) + fabsf(b)), 0.f);
        return dd * dd * p.c > CULL_EXPONENT;
    }
}

// The active points of a warp as one test (slope model): the smallest box
// [t0lo, t0hi] x [t1lo, t1hi] holding them.  Its distance to a block's box
// is at most each point's own (every rounding is monotone), so a block this
// test skips is skipped by each point's box_culled: the kept set is a
// superset of the union of the points' own, and the extra blocks add exact
// zeros to each sum.  One test instead of one per point; the points of a
// warp are spatial neighbours (sorted seeds), so few blocks are added.
struct CullSpan {
    float t0lo, t0hi, t1lo, t1hi, c;
};
template <int P>
__device__ __forceinline__ CullSpan cull_span(const float (&t0)[P], const float (&t1)[P], const bool (&act)[P],
                                              float cull) {
    CullSpan s{INFINITY, -INFINITY, INFINITY, -INFINITY, cull};
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!act[p]) continue;
        if (!(isfinite(t0[p]) && isfinite(t1[p]))) s.c = INFINITY;  // never skip around a non-finite point
        s.t0lo = fminf(s.t0lo, t0[p]);
        s.t0hi = fmaxf(s.t0hi, t0[p]);
        s.t1lo = fminf(s.t1lo, t1[p]);
        s.t1hi = fmaxf(s.t1hi, t1[p]);
    }
    return s;
}
__device__ __forceinline__ bool span_culled(const float4 A, const float w, const CullSpan &s) {
    const float du = fmaxf(fmaxf(A.x - s.t0hi, s.t0lo - A.y), 0.f);
    const float dv = fmaxf(fmaxf(A.z - s.t1hi, s.t1lo - A.w), 0.f);
    return __fmaf_rn(du, du, dv * dv) * w > s.c;
}

// Pass over the hits that can contribute for the P points of the warp.
// Without boxes it is for_each_hit.  With boxes, each chunk of KEPT_CHUNK
// blocks is tested (lane l tests blocks l, l + 32, l + 64, l + 96 of the
// chunk in turn, or, for a chunk of staged slope-model boxes, superblock l
// first and then the blocks of the kept superblocks), the ballots append
// the blocks some point needs, in increasing order, as offsets to the warp's
// list (consecutive chunks while they fit), and the warp walks the list,
// lane l taking hit 32 b + l of each block: the same per-lane order as the full pass minus blocks whose terms
// are all exactly zero - so every sum is bitwise the full pass's sum.
// With REUSE, reuse >= 0 walks list[0 .. reuse) as an earlier pass left it,
// without tests (the caller knows it holds every block this pass needs), and
// reuse == -2 reports through built the number of kept blocks when one walk
// held them all (else -1).  Returns the hits visited (for the work counters).
template <int MODEL, int UNROLL = 2, bool REUSE = false, typename T, typename F, typename F2>
__device__ __forceinline__ int hit_pass(const float4 *__restrict__ sh, const float4 *__restrict__ gh, int n_staged,
                                        int H, int lane, const float4 *__restrict__ sbox, const float *__restrict__ sz2,
                                        const float4 *__restrict__ ssb, const float *__restrict__ ssz2,
                                        const float4 *__restrict__ gbox, int n_sbox, int *__restrict__ list,
                                        T &&needed, F &&f, F2 &&f2, int reuse = -1, int *built = nullptr) {
    if (!gbox) {
        for_each_hit(sh, gh, n_staged, H, lane, f, f2);
        return H;
    }
    int visited = 0;
    const int nblk = (H + 31) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int *slot = list + KEPT_CHUNK;  // the warp's 32 superblock slots
    // Kept blocks of consecutive chunks collect in the list (increasing block
    // order) as long as a chunk's candidates are sure to fit; then the list
    // is walked once - usually a single walk per pass.
    int c0 = 0, walks = 0, first = -1;
    for (;;) {
        int cnt = 0;
        bool done = false;
        if (REUSE && reuse >= 0) {  // the list an earlier pass built
            cnt = reuse;
            done = true;
        } else for (;;) {
            if (c0 >= nblk) {
                done = true;
                break;
            }
            if (MODEL == RETINA_VELO_SLOPES && c0 + KEPT_CHUNK <= n_sbox) {
                // two levels: lane l tests superblock c0 / 4 + l (blocks 4 of them),
                // then the blocks of the superblocks some point needs, in
                // increasing order (superblock rank, block within it)
                const int q = (c0 >> 2) + lane;
                const bool keep_q = needed(ssb[q], ssz2[q]);
                const unsigned mq = __ballot_sync(0xffffffffu, keep_q);
                const int n_sub = 4 * __popc(mq);
                if (cnt + n_sub > KEPT_CHUNK) break;  // walk the list first, then test this chunk again
                c0 += KEPT_CHUNK;
                if (mq == 0u) continue;
                if (keep_q) slot[__popc(mq & lt)] = q;
                __syncwarp();
                for (int k0 = 0; k0 < n_sub; k0 += 32) {
                    const int k = k0 + lane;
                    bool keep = false;
                    int b = 0;
                    if (k < n_sub) {
                        b = 4 * slot[k >> 2] + (k & 3);
                        keep = needed(sbox[b], sz2[b]);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) list[cnt + __popc(m & lt)] = b * 32;
                    cnt += __popc(m);
                }
                __syncwarp();  // the slots are rewritten by the next chunk
            } else {
                const int n_chunk = nblk - c0 < KEPT_CHUNK ? nblk - c0 : KEPT_CHUNK;
                if (cnt + n_chunk > KEPT_CHUNK) break;  // walk the list first
#pragma unroll 1
                for (int w = 0; w < KEPT_CHUNK / 32 && 32 * w < n_chunk; ++w) {
                    const int b = c0 + 32 * w + lane;
                    bool keep = false;
                    if (b < nblk) {
                        float4 A;
                        float z2;
                        if (b < n_sbox) {
                            A = sbox[b];
                            z2 = sz2[b];
                        } else {
                            A = __ldg(gbox + 2 * b);
                            z2 = search_box<MODEL>(A, __ldg(gbox + 2 * b + 1));
                        }
                        keep = needed(A, z2);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) list[cnt + __popc(m & lt)] = b * 32;
                    cnt += __popc(m);
                }
                c0 += KEPT_CHUNK;
            }
        }
        __syncwarp();
        if (cnt > 0) {
            // hits visited: 32 per kept block, the event's last block holding H - 32 (nblk - 1)
            const int last = list[cnt - 1];
            visited += 32 * cnt - (last == 32 * (nblk - 1) ? 32 * nblk - H : 0);
            // One loop body for every kept block (the kernel is large enough that
            // its instruction footprint, not its instruction count, sets the
            // pace: a second copy of the pair arithmetic doubled the instruction
            // fetch stalls).  Blocks held whole in shared memory form a prefix of
            // the list and are read from there, the rest from global memory
            // through the same generic pointer (a staged hit is the same value in
            // both places); the event's last block, when partial, is left to the
            // one-block remainder, whose lanes past the event add nothing.  Per
            // lane the hits are added in list order, and f2(a, b) adds exactly
            // what f(a); f(b) adds, so every sum is the full pass's.
            int n_fast = cnt;  // the staged prefix of the list
            if (last + 32 > n_staged) {
                n_fast = 0;
                for (int k0 = 0; k0 < cnt; k0 += 32) {
                    const int k = k0 + lane;
                    n_fast += __popc(__ballot_sync(0xffffffffu, k < cnt && list[k] + 32 <= n_staged));
                }
            }
            const int n_pairs_end = cnt - ((last == 32 * (nblk - 1) && (H & 31)) ? 1 : 0);
            int i = 0;
#pragma unroll 1
            for (int seg = 0; seg < 2; ++seg) {
                const float4 *src = seg == 0 ? sh : gh;
                const int end = seg == 0 ? (n_fast < n_pairs_end ? n_fast : n_pairs_end) : n_pairs_end;
#pragma unroll 1
                for (; i + UNROLL <= end; i += UNROLL) {
                    // UNROLL = 4 (one point per warp, latency-bound): four blocks in flight
                    const float4 ha = src[list[i] + lane], hb = src[list[i + 1] + lane];
                    if (UNROLL == 4) {
                        const float4 hc = src[list[i + 2] + lane], hd = src[list[i + 3] + lane];
                        f2(ha, hb);
                        f2(hc, hd);
                    } else {
                        f2(ha, hb);
                    }
                }
                if (UNROLL == 4 && i + 2 <= end) {
                    f2(src[list[i] + lane], src[list[i + 1] + lane]);
                    i += 2;
                }
            }
#pragma unroll 1
            for (; i < cnt; ++i) {
                const int k = list[i] + lane;
                const float4 *src = list[i] + 32 <= n_staged ? sh : gh;  // a staged remainder from shared memory
                if (k < H) f(src[k]);
            }
            __syncwarp();  // the list is rewritten by the next round
        }
        if constexpr (REUSE) {
            if (walks++ == 0) first = cnt;
        }
        if (done) break;
    }
    if constexpr (REUSE) {
        if (built) *built = (reuse == -2 && walks == 1) ? first : -1;  // the whole kept set, if one walk held it
    }
    return visited;
}

// Algorithm 1 for one seed per warp (the latency-bound shape), with the same
// arithmetic as search_group<MODEL, 1> in fewer passes: the first line-search
// trial of update j (t = 1) is the point update j + 1 starts from whenever it
// is accepted - 91 % of the time on the VELO-like events - so that pass also
// accumulates the gradient/Hessian sums at bandwidth sigma_{j+1}, and update
// j + 1 uses them instead of a pass of its own.  The pass skips a block only
// when it is skippable at both bandwidths, so each sum gets exactly the terms
// of its own pass plus exact zeros, in the same per-lane order: every result,
// status and trial count is bitwise search_group's.
template <int MODEL, int UPD = RETINA_UPDATE_TRUNCATED_NEWTON>
__device__ __forceinline__ void search_one(const float4 *__restrict__ sh, const float4 *__restrict__ gh, int n_staged,
                                           int H, int lane, const float4 *__restrict__ sbox, const float *__restrict__ sz2,
                                           const float4 *__restrict__ ssb, const float *__restrict__ ssz2,
                                           const float4 *__restrict__ gbox, int n_sbox, int *__restrict__ list,
                                           const float *__restrict__ seeds, const LsParams &prm,
                                           float *__restrict__ theta_out, float *__restrict__ R_out,
                                           uint8_t *__restrict__ status, uint8_t *__restrict__ n_evals,
                                           unsigned long long *__restrict__ work) {
    uint32_t w_rgh = 0, w_r = 0;  // hits visited (fewer than 2^32 per seed)
    constexpr int NS = Model<MODEL>::NS;
    float th0 = seeds[0], th1 = seeds[1], Rfin = 0.f;
    int evals = 0;
    bool failed = false;
    float S[NS];
    bool have = false;  // S holds the sums at (theta, sigma_j) from the previous update's first trial
    for (int j = 0; j < prm.q; ++j) {
        const float kk = prm.kk[j], k = prm.k[j], cull = prm.cull[j];
        if (!have) {
            RghAcc<MODEL> acc;
            acc.zero();
            const CullPt cp = cull_pt<MODEL>(th0, th1, kk, cull);
            const int vis = hit_pass<MODEL, 4>(
                sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list,
                [&](const float4 A, const float z2) { return !box_culled<MODEL>(A, z2, cp); },
                [&](const float4 h) { acc.add(h, th0, th1, kk); },
                [&](const float4 a, const float4 b) { acc.add2(a, b, th0, th1, kk); });
            acc.sums(S);
#pragma unroll
            for (int i = 0; i < NS; ++i) S[i] = warp_sum(S[i]);
            w_rgh += (uint32_t)vis;
        }
        have = false;
        float R, g0, g1, H00, H01, H11, pp0, pp1;
        sums_to_rgh<MODEL>(S, k, R, g0, g1, H00, H01, H11);
        update_direction<UPD>(g0, g1, H00, H01, H11, pp0, pp1);
        cap_step(pp0, pp1, prm.box.step0, prm.box.step1, prm.cap);
        const float slope = dir_slope(g0, g1, pp0, pp1);
        float t = 1.f;
        bool pending = true;
        Rfin = R;  // R at the point if no step is accepted
        const bool fuse = j + 1 < prm.q;
        // the first trial (t = 1) alone; once it is rejected, with
        // prm.pair_trials, the trials t and t / 2 share one pass (a block is skipped only when both points skip
        // it, so each R is bitwise its own pass's) and are tested in order:
        // the accepted point, its R and the trial count are the sequential
        // backtracking's, in about half the dependent passes
        for (int hv = 0; hv <= prm.max_halvings && pending;) {
            const float tr0 = __fmaf_rn(t, pp0, th0), tr1 = __fmaf_rn(t, pp1, th1);
            // (compiled into the truncated Newton search only: the comparison
            // updates run throughput-bound batches, where the extra pass body
            // would only crowd the instruction cache)
            constexpr bool PAIRS = UPD == RETINA_UPDATE_TRUNCATED_NEWTON;
            const bool two = PAIRS && prm.pair_trials && hv > 0 && hv + 1 <= prm.max_halvings;
            const float tb = t * 0.5f;
            const float tb0 = __fmaf_rn(tb, pp0, th0), tb1 = __fmaf_rn(tb, pp1, th1);
            float Rt = 0.f, Rb = 0.f;
            int vis;
            if (hv == 0 && fuse) {
                const float kk2 = prm.kk[j + 1];
                const CullPt ct = cull_pt_union<MODEL>(tr0, tr1, kk, cull, kk2, prm.cull[j + 1]);
                RghAcc<MODEL> acc;
                acc.zero();
                vis = hit_pass<MODEL, 4>(
                    sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list,
                    [&](const float4 A, const float z2) { return !box_culled<MODEL>(A, z2, ct); },
                    [&](const float4 h) {
                        Rt = __fadd_rn(Rt, pair_r<MODEL>(h, tr0, tr1, kk));
                        acc.add(h, tr0, tr1, kk2);
                    },
                    [&](const float4 a, const float4 b) {
                        pair_r2<MODEL>(a, b, tr0, tr1, kk, Rt);
                        acc.add2(a, b, tr0, tr1, kk2);
                    });
                acc.sums(S);
                w_rgh += (uint32_t)vis;
            } else if (PAIRS && two) {
                const CullPt ca = cull_pt<MODEL>(tr0, tr1, kk, cull), cb = cull_pt<MODEL>(tb0, tb1, kk, cull);
                auto need2 = [&](const float4 A, const float z2) {
                    return !box_culled<MODEL>(A, z2, ca) || !box_culled<MODEL>(A, z2, cb);
                };
                if constexpr (MODEL == RETINA_VELO_SLOPES) {
                    // both trial points in packed FP32x2 (bitwise pair_r per lane)
                    const unsigned long long nt0 = pack2(-tr0, -tb0), nt1 = pack2(-tr1, -tb1);
                    const unsigned long long nkk = pack2(-kk, -kk);
                    unsigned long long Rt2 = 0ull;
                    vis = hit_pass<MODEL, 4>(
                        sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, need2,
                        [&](const float4 h) { pair_r_x2(h, nt0, nt1, nkk, Rt2); },
                        [&](const float4 a, const float4 b) {
                            pair_r_x2(a, nt0, nt1, nkk, Rt2);
                            pair_r_x2(b, nt0, nt1, nkk, Rt2);
                        });
                    unpack2(Rt2, Rt, Rb);
                } else {
                    vis = hit_pass<MODEL, 4>(
                        sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, need2,
                        [&](const float4 h) {
                            Rt = __fadd_rn(Rt, pair_r<MODEL>(h, tr0, tr1, kk));
                            Rb = __fadd_rn(Rb, pair_r<MODEL>(h, tb0, tb1, kk));
                        },
                        [&](const float4 a, const float4 b) {
                            pair_r2<MODEL>(a, b, tr0, tr1, kk, Rt);
                            pair_r2<MODEL>(a, b, tb0, tb1, kk, Rb);
                        });
                }
                w_r += (uint32_t)vis;  // the second point's pairs
            } else {
                const CullPt ct = cull_pt<MODEL>(tr0, tr1, kk, cull);
                vis = hit_pass<MODEL, 4>(
                    sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list,
                    [&](const float4 A, const float z2) { return !box_culled<MODEL>(A, z2, ct); },
                    [&](const float4 h) { Rt = __fadd_rn(Rt, pair_r<MODEL>(h, tr0, tr1, kk)); },
                    [&](const float4 a, const float4 b) { pair_r2<MODEL>(a, b, tr0, tr1, kk, Rt); });
            }
            w_r += (uint32_t)vis;
            ++evals;
            const float rt = warp_sum(Rt);
            if (rt >= armijo_bound(R, prm.c1, t, slope)) {
                th0 = tr0;
                th1 = tr1;
                Rfin = rt;  // R at the accepted point, this update's bandwidth
                pending = false;
                if (hv == 0 && fuse) {
#pragma unroll
                    for (int i = 0; i < NS; ++i) S[i] = warp_sum(S[i]);
                    have = true;  // the next update's sums at the accepted point
                }
            } else if (two) {
                ++evals;
                const float rb = warp_sum(Rb);
                if (rb >= armijo_bound(R, prm.c1, tb, slope)) {
                    th0 = tb0;
                    th1 = tb1;
                    Rfin = rb;
                    pending = false;
                } else {
                    t = tb * 0.5f;
                }
                hv += 2;
            } else {
                t *= 0.5f;
                ++hv;
            }
        }
        if (pending) failed = true;
    }
    if (work && lane == 0) {
        atomicAdd(work + RETINA_WORK_RGH, (unsigned long long)w_rgh);
        atomicAdd(work + RETINA_WORK_R, (unsigned long long)w_r);
    }
    if (lane != 0) return;
    const float hi0 = prm.box.lo0 + (float)prm.box.n0 * prm.box.step0;
    const float hi1 = prm.box.lo1 + (float)prm.box.n1 * prm.box.step1;
    uint8_t st;
    if (!(isfinite(th0) && isfinite(th1) && isfinite(Rfin)))
        st = 3;
    else if (!(th0 >= prm.box.lo0 && th0 < hi0 && th1 >= prm.box.lo1 && th1 < hi1))
        st = 2;
    else
        st = failed ? 1 : 0;
    theta_out[0] = th0;
    theta_out[1] = th1;
    R_out[0] = Rfin;
    status[0] = st;
    if (n_evals) n_evals[0] = (uint8_t)(evals < 255 ? evals : 255);
}

// Warp totals of the seven RGH sums of four points (packed pairs A: points 0
// and 1, B: points 2 and 3, per lane), reduced and scattered at once: lane l
// ends with the total of sum l & 7 of point l >> 3 (0.0 for l & 7 = 7).  Each
// level halves what a lane holds - it keeps the half its lane bit selects and
// adds the partner's copy of that half - in warp_sum's order (xor 16, 8, 4, 2,
// 1), and every partial it adds is the one warp_sum adds at that level, so
// each total is bitwise warp_sum's: 28 shuffles for the 28 totals instead of
// 140.
__device__ __forceinline__ float scatter_sums4(const unsigned long long (&A)[7], const unsigned long long (&B)[7],
                                               int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
    float v[8];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const unsigned long long got = __shfl_xor_sync(0xffffffffu, b4 ? A[i] : B[i], 16);
        float lo, hi;
        unpack2(add2_rn(b4 ? B[i] : A[i], got), lo, hi);
        v[i] = __fadd_rn(b3 ? hi : lo, __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8));
    }
    v[7] = 0.f;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = __fadd_rn(b2 ? v[4 + i] : v[i], __shfl_xor_sync(0xffffffffu, b2 ? v[i] : v[4 + i], 4));
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        x[i] = __fadd_rn(b1 ? w[2 + i] : w[i], __shfl_xor_sync(0xffffffffu, b1 ? w[i] : w[2 + i], 2));
    return __fadd_rn(b0 ? x[1] : x[0], __shfl_xor_sync(0xffffffffu, b0 ? x[0] : x[1], 1));
}

// Warp totals of one sum of four points (packed pairs A: points 0, 1, B:
// points 2, 3): every lane of group l >> 3 ends with point l >> 3's total,
// bitwise warp_sum's (the same levels as scatter_sums4, then xor 4, 2, 1).
__device__ __forceinline__ float group_sums4(unsigned long long A, unsigned long long B, int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float lo, hi;
    unpack2(add2_rn(b4 ? B : A, __shfl_xor_sync(0xffffffffu, b4 ? A : B, 16)), lo, hi);
    float v = __fadd_rn(b3 ? hi : lo, __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8));
#pragma unroll
    for (int m = 4; m >= 1; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
    return v;
}

// Algorithm 1 for the P seeds of one warp: q truncated-Newton updates
// (gradient/Hessian pass, Newton-CG direction, step cap, Armijo backtracking
// at bandwidth sigma_j), then R(theta_q; sigma_q), status and the number of
// R-only passes.  seeds / outputs point at the group's first seed; only the
// first n_live (<= P) seeds exist.  Warp-uniform control flow throughout.
// The per-point state of search_group kept across passes.
template <int P>
struct GroupState {
    float th0[P], th1[P], Rfin[P], R[P], pp0[P], pp1[P], slope[P], t[P];
    int evals[P];
    bool live[P], failed[P], pending[P];
};

template <int MODEL, int P, int UPD = RETINA_UPDATE_TRUNCATED_NEWTON, bool SS = false, bool RL = false>
__device__ __forceinline__ void search_group(const float4 *__restrict__ sh, const float4 *__restrict__ gh,
                                             int n_staged, int H, int lane, const float4 *__restrict__ sbox,
                                             const float *__restrict__ sz2, const float4 *__restrict__ ssb,
                                             const float *__restrict__ ssz2, const float4 *__restrict__ gbox,
                                             int n_sbox, int *__restrict__ list,
                                             const float *__restrict__ seeds,
                                             int n_live, const LsParams &prm, float *__restrict__ theta_out,
                                             float *__restrict__ R_out, uint8_t *__restrict__ status,
                                             uint8_t *__restrict__ n_evals, unsigned long long *__restrict__ work,
                                             GroupState<P> *state = nullptr) {
    if constexpr (P == 1) {
        search_one<MODEL, UPD>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, seeds, prm, theta_out, R_out,
                          status, n_evals, work);
        return;
    }
    uint32_t w_rgh = 0, w_r = 0;  // (point, hit) pairs visited (fewer than 2^32 per group)
    constexpr int NS = Model<MODEL>::NS;
    // the points' state between passes: warp-uniform, in registers, or (SS)
    // once per warp in shared memory, where 32 lanes' copies would spill
    static_assert(!SS || (P == 4 && MODEL == RETINA_VELO_SLOPES), "shared state: four slope-model points");
    GroupState<P> gs_local;
    GroupState<P> &gs = SS ? *state : gs_local;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        gs.live[p] = p < n_live;
        const int o = (gs.live[p] ? p : 0) * 2;
        gs.th0[p] = seeds[o];
        gs.th1[p] = seeds[o + 1];
        gs.failed[p] = false;
        gs.evals[p] = 0;
        gs.Rfin[p] = 0.f;
    }

    for (int j = 0; j < prm.q; ++j) {
        const float kk = prm.kk[j], k = prm.k[j], cull = prm.cull[j];
        // (R, g, H) at the current points
        RghAcc<MODEL> acc[P];
        CullPt cp[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            acc[p].zero();
            cp[p] = cull_pt<MODEL>(gs.th0[p], gs.th1[p], kk, cull);
        }
        CullSpan span = cull_span<P>(gs.th0, gs.th1, gs.live, cull);
        // RL (packed slope-model groups on events of one 128-block chunk,
        // where each box test is one block per lane, with no superblocks):
        // this pass tests its blocks against the points' box grown by one
        // capped step - every trial point of the update lies inside it
        // (|p_a| <= cap step_a, t <= 1; the 0.1 % covers the roundings) - so
        // that the list, when one walk holds it, serves all the update's
        // trials without tests; the extra blocks add exact zeros.
        int kept = -1;
        bool reuse = false;
        if constexpr (RL) {
            static_assert(P % 2 == 0 && MODEL == RETINA_VELO_SLOPES, "packed slope-model groups");
            reuse = ((H + 31) >> 5) <= KEPT_CHUNK;
            const float g = reuse ? 1.001f * prm.cap : 0.f;
            const float d0 = g * prm.box.step0, d1 = g * prm.box.step1;
            span.t0lo -= d0;
            span.t0hi += d0;
            span.t1lo -= d1;
            span.t1hi += d1;
        }
        auto needed = [&](const float4 A, const float z2) {
            if constexpr (P % 2 == 0 && MODEL == RETINA_VELO_SLOPES) return !span_culled(A, z2, span);
            bool need = false;
#pragma unroll
            for (int p = 0; p < P; ++p) need |= gs.live[p] && !box_culled<MODEL>(A, z2, cp[p]);
            return need;
        };
        float S[P][NS];
        float tot_ss = 0.f;  // four points: this lane's scattered total
        int vis;
        if constexpr (P % 2 == 0 && MODEL == RETINA_VELO_SLOPES) {
            // the points' sums in packed FP32x2, two points per register pair
            // (bitwise the scalar sums)
            constexpr int NP = P / 2;
            RghAcc2 a2[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                a2[q].set(gs.th0[2 * q], gs.th1[2 * q], gs.th0[2 * q + 1], gs.th1[2 * q + 1], kk);
                a2[q].zero();
            }
            vis = hit_pass<MODEL, 2, RL>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, needed,
                                  [&](const float4 h) {
#pragma unroll
                                      for (int q = 0; q < NP; ++q) a2[q].add(h);
                                  },
                                  [&](const float4 a, const float4 b) {
#pragma unroll
                                      for (int q = 0; q < NP; ++q) {
                                          a2[q].add(a);
                                          a2[q].add(b);
                                      }
                                  },
                                  reuse ? -2 : -1, &kept);
            if constexpr (SS) {
                tot_ss = scatter_sums4(a2[0].S, a2[1].S, lane);
            } else {
#pragma unroll
                for (int q = 0; q < NP; ++q) a2[q].sums(S[2 * q], S[2 * q + 1]);
            }
        } else {
            vis = hit_pass<MODEL>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, needed,
                                          [&](const float4 h) {
#pragma unroll
                                              for (int p = 0; p < P; ++p) acc[p].add(h, gs.th0[p], gs.th1[p], kk);
                                          },
                                          [&](const float4 a, const float4 b) {
#pragma unroll
                                              for (int p = 0; p < P; ++p) acc[p].add2(a, b, gs.th0[p], gs.th1[p], kk);
                                          });
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p].sums(S[p]);
        }
        w_rgh += (uint32_t)vis * (uint32_t)n_live;
        if constexpr (SS) {
            // four points (state in shared memory): the 28 totals scattered
            // over the warp, then lanes 8p .. 8p + 7 take point p's update
            // together - one copy of the update code for all four points
            const float tot = tot_ss;
            const int p = lane >> 3;
            float Sp[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) Sp[i] = __shfl_sync(0xffffffffu, tot, (lane & 24) | i);
            float R, g0, g1, H00, H01, H11, pp0, pp1;
            sums_to_rgh<MODEL>(Sp, k, R, g0, g1, H00, H01, H11);
            update_direction<UPD>(g0, g1, H00, H01, H11, pp0, pp1);
            cap_step(pp0, pp1, prm.box.step0, prm.box.step1, prm.cap);
            const float slope = dir_slope(g0, g1, pp0, pp1);
            if ((lane & 7) == 0) {
                gs.R[p] = R;
                gs.pp0[p] = pp0;
                gs.pp1[p] = pp1;
                gs.slope[p] = slope;
                gs.t[p] = 1.f;
                gs.pending[p] = gs.live[p];
                gs.Rfin[p] = R;  // R at the point if no step is accepted
            }
            __syncwarp();
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) {
#pragma unroll
                for (int i = 0; i < NS; ++i) S[p][i] = warp_sum(S[p][i]);
                float g0, g1, H00, H01, H11;
                sums_to_rgh<MODEL>(S[p], k, gs.R[p], g0, g1, H00, H01, H11);
                update_direction<UPD>(g0, g1, H00, H01, H11, gs.pp0[p], gs.pp1[p]);
                cap_step(gs.pp0[p], gs.pp1[p], prm.box.step0, prm.box.step1, prm.cap);
                gs.slope[p] = dir_slope(g0, g1, gs.pp0[p], gs.pp1[p]);
                gs.t[p] = 1.f;
                gs.pending[p] = gs.live[p];
                gs.Rfin[p] = gs.R[p];  // R at the point if no step is accepted
            }
        }
        // backtracking line search, all pending seeds of the warp together
        for (int hv = 0; hv <= prm.max_halvings; ++hv) {
            bool any = false;
#pragma unroll
            for (int p = 0; p < P; ++p) any |= gs.pending[p];
            if (!any) break;
            float tr0[P], tr1[P], Rt[P];
            CullPt ct[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                tr0[p] = __fmaf_rn(gs.t[p], gs.pp0[p], gs.th0[p]);
                tr1[p] = __fmaf_rn(gs.t[p], gs.pp1[p], gs.th1[p]);
                Rt[p] = 0.f;
                ct[p] = cull_pt<MODEL>(tr0[p], tr1[p], kk, cull);
            }
            const CullSpan span_r = cull_span<P>(tr0, tr1, gs.pending, cull);
            auto needed_r = [&](const float4 A, const float z2) {
                if constexpr (P % 2 == 0 && MODEL == RETINA_VELO_SLOPES) return !span_culled(A, z2, span_r);
                bool need = false;
#pragma unroll
                for (int p = 0; p < P; ++p) need |= gs.pending[p] && !box_culled<MODEL>(A, z2, ct[p]);
                return need;
            };
            float rt_ss = 0.f;  // four points: the total of this lane's point
            int vis;
            if constexpr (P % 2 == 0 && MODEL == RETINA_VELO_SLOPES) {
                // the trial points in packed FP32x2, two per register pair; a
                // point whose line search is over accumulates too, and its sum
                // is not used
                constexpr int NP = P / 2;
                unsigned long long nt0[NP], nt1[NP], Rt2[NP];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    nt0[q] = pack2(-tr0[2 * q], -tr0[2 * q + 1]);
                    nt1[q] = pack2(-tr1[2 * q], -tr1[2 * q + 1]);
                    Rt2[q] = 0ull;
                }
                const unsigned long long nkk = pack2(-kk, -kk);
                vis = hit_pass<MODEL, 2, RL>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list,
                                      needed_r,
                                      [&](const float4 h) {
#pragma unroll
                                          for (int q = 0; q < NP; ++q) pair_r_x2(h, nt0[q], nt1[q], nkk, Rt2[q]);
                                      },
                                      [&](const float4 a, const float4 b) {
#pragma unroll
                                          for (int q = 0; q < NP; ++q) {
                                              pair_r_x2(a, nt0[q], nt1[q], nkk, Rt2[q]);
                                              pair_r_x2(b, nt0[q], nt1[q], nkk, Rt2[q]);
                                          }
                                      },
                                      kept);
                if constexpr (SS) {
                    rt_ss = group_sums4(Rt2[0], Rt2[1], lane);
                } else {
#pragma unroll
                    for (int q = 0; q < NP; ++q) unpack2(Rt2[q], Rt[2 * q], Rt[2 * q + 1]);
                }
            } else {
                vis = hit_pass<MODEL>(sh, gh, n_staged, H, lane, sbox, sz2, ssb, ssz2, gbox, n_sbox, list, needed_r,
                                              [&](const float4 h) {
#pragma unroll
                                                  for (int p = 0; p < P; ++p)
                                                      if (gs.pending[p])
                                                          Rt[p] = __fadd_rn(Rt[p], pair_r<MODEL>(h, tr0[p], tr1[p], kk));
                                              },
                                              [&](const float4 a, const float4 b) {
#pragma unroll
                                                  for (int p = 0; p < P; ++p)
                                                      if (gs.pending[p]) pair_r2<MODEL>(a, b, tr0[p], tr1[p], kk, Rt[p]);
                                              });
            }
            int n_pend = 0;
#pragma unroll
            for (int p = 0; p < P; ++p) n_pend += gs.pending[p] ? 1 : 0;
            w_r += (uint32_t)vis * (uint32_t)n_pend;
            if constexpr (SS) {
                // lanes 8p .. 8p + 7 test point p's trial; lane 8p writes
                const int p = lane >> 3;
                const bool pend = gs.pending[p];
                const float t = gs.t[p];
                const bool acc = pend && rt_ss >= armijo_bound(gs.R[p], prm.c1, t, gs.slope[p]);
                const float a0 = __fmaf_rn(t, gs.pp0[p], gs.th0[p]), a1 = __fmaf_rn(t, gs.pp1[p], gs.th1[p]);
                __syncwarp();  // every lane has read the state it needs
                if (pend && (lane & 7) == 0) {
                    ++gs.evals[p];
                    if (acc) {
                        gs.th0[p] = a0;  // the trial point (bitwise tr0, tr1)
                        gs.th1[p] = a1;
                        gs.Rfin[p] = rt_ss;  // R at the accepted point, this update's bandwidth
                        gs.pending[p] = false;
                    } else {
                        gs.t[p] = __fmul_rn(t, 0.5f);
                    }
                }
                __syncwarp();
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (!gs.pending[p]) continue;
                    ++gs.evals[p];
                    const float rt = warp_sum(Rt[p]);
                    if (rt >= armijo_bound(gs.R[p], prm.c1, gs.t[p], gs.slope[p])) {
                        gs.th0[p] = tr0[p];
                        gs.th1[p] = tr1[p];
                        gs.Rfin[p] = rt;  // R at the accepted point, this update's bandwidth
                        gs.pending[p] = false;
                    } else {
                        gs.t[p] *= 0.5f;
                    }
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (gs.pending[p]) gs.failed[p] = true;
    }

    // After the last update Rfin holds R(theta_q; sigma_q): the accepted
    // trial's response, or the response at the unmoved point - the same sum,
    // in the same order, that a separate evaluation would produce.
    if (work && lane == 0) {
        atomicAdd(work + RETINA_WORK_RGH, (unsigned long long)w_rgh);
        atomicAdd(work + RETINA_WORK_R, (unsigned long long)w_r);
    }
    const float hi0 = prm.box.lo0 + (float)prm.box.n0 * prm.box.step0;
    const float hi1 = prm.box.lo1 + (float)prm.box.n1 * prm.box.step1;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!gs.live[p] || lane != 0) continue;
        uint8_t st;
        if (!(isfinite(gs.th0[p]) && isfinite(gs.th1[p]) && isfinite(gs.Rfin[p])))
            st = 3;
        else if (!(gs.th0[p] >= prm.box.lo0 && gs.th0[p] < hi0 && gs.th1[p] >= prm.box.lo1 && gs.th1[p] < hi1))
            st = 2;
        else
            st = gs.failed[p] ? 1 : 0;
        theta_out[2 * p] = gs.th0[p];
        theta_out[2 * p + 1] = gs.th1[p];
        R_out[p] = gs.Rfin[p];
        status[p] = st;
        if (n_evals) n_evals[p] = (uint8_t)(gs.evals[p] < 255 ? gs.evals[p] : 255);
    }
}

}  // namespace retina
