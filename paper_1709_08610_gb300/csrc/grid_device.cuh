// Exact block skipping shared by the grid-response kernels (CUDA-core and
// tensor-core contractions).
#pragma once

#include "internal.cuh"

namespace retina {

// Exact skipping of hit blocks for a whole tile of cells (boxes from
// retina_prepare_hits): the lower bound, over the tile's parameter range and
// the block's box, of the exponent s^2 log2(e) / sigma^2 (or of one axis's
// part of it for the separable panels) must exceed GRID_CULL_EXPONENT, so
// that every skipped ex2.approx.ftz value is exactly zero (x > 126; 140
// leaves a margin, and a relative slack of 1e-6 per magnitude covers the
// rounding of the bound).  Non-finite boxes are never skipped.
constexpr float GRID_CULL_EXPONENT = 140.f;

// Distance between the intervals [al, ah] and [bl, bh], minus a rounding
// slack of 1e-6 per magnitude; 0 when they overlap.
__device__ __forceinline__ float gap_ii(float al, float ah, float bl, float bh) {
    const float d = fmaxf(fmaxf(bl - ah, al - bh), 0.f);
    return fmaxf(d - 1e-6f * (fabsf(al) + fabsf(ah) + fabsf(bl) + fabsf(bh)), 0.f);
}

struct TileRange {
    float t0l, t0h, t1l, t1h;  // cell-centre range of the tile's valid cells
};

__device__ __forceinline__ TileRange tile_range(const GridDev &g, int ti0, int tj0, int w0, int w1) {
    const int i1 = (ti0 + w0 - 1 < g.n0 - 1) ? ti0 + w0 - 1 : g.n0 - 1;
    const int j1 = (tj0 + w1 - 1 < g.n1 - 1) ? tj0 + w1 - 1 : g.n1 - 1;
    return TileRange{cell_centre(g.lo0, g.step0, ti0), cell_centre(g.lo0, g.step0, i1),
                     cell_centre(g.lo1, g.step1, tj0), cell_centre(g.lo1, g.step1, j1)};
}

// Slope-model boxes (umin, umax, vmin, vmax | |z|min, |z|max): for every
// cell of the tile and hit of the block, (x - t_x z)^2 = z^2 (u - t_x)^2 >=
// |z|min^2 gap(t_x range, u range)^2, likewise for y.  Separable panels are
// all zero when either axis alone exceeds the cut.
__device__ __forceinline__ bool block_zero_sep(const float4 A, const float4 B, const TileRange &r, float kk) {
    if (!isfinite(B.x)) return false;
    const float du = gap_ii(r.t0l, r.t0h, A.x, A.y), dv = gap_ii(r.t1l, r.t1h, A.z, A.w);
    const float z2k = B.x * B.x * kk;
    return du * du * z2k > GRID_CULL_EXPONENT || dv * dv * z2k > GRID_CULL_EXPONENT;
}

// The tensor-core contraction (grid_tc.cu) on tiles of 128 x bn cells (bn =
// 128 or 256), launched with programmatic serialization on stream st.
cudaError_t launch_grid_tc(int bn, dim3 grid, cudaStream_t st, const float4 *hits, int64_t n_hits, const int64_t *off,
                           const float4 *boxes, GridDev g, float kk, int splits, int tiles0, float *out,
                           int64_t split_stride, int64_t event_stride, int32_t *err);

}  // namespace retina
