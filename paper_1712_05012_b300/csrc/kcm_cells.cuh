// Mixed-mode cell arithmetic of the binning kernels (kcm_kernels.cu, kcm_bin_cluster.cu): the cell of a
// centre and its offset from the cell corner, from the double-float centres and the grid origin as an
// exact double-float, rounded once to float. On the FP32 pipe only: on B300 an FP64 warp instruction
// holds a sub-partition's FP64 pipe for ~84 cycles. (FP64 mode rounds the FP64 difference instead; the
// two can differ by one float rounding, which the cell margin absorbs.)
#pragma once

#include "kcm_df.cuh"
#include "kcm_device.h"

namespace kcm {
namespace dev {

// cell index along one axis: the offset from the origin o times the inverse edge, clamped to [0, n)
__device__ __forceinline__ int mixed_cell_axis(df p, float2 o, float inv_sf, int n) {
    return min(max((int)floorf(sub(p, df{o.x, o.y}).hi * inv_sf), 0), n - 1);
}

// offset from the corner of cell c along one axis (origin + c s; the product c s is exact as a
// double-float, s being a multiple of 2^-10 exact in float)
__device__ __forceinline__ float mixed_offset(df p, float2 o, int c, float sf) {
    return sub(sub(p, df{o.x, o.y}), mul(df{(float)c, 0.0f}, df{sf, 0.0f})).hi;
}

// a > b for normalized double-floats (their order-preserving keys)
__device__ __forceinline__ bool df_gt(df a, df b) { return dfkey(a) > dfkey(b); }

// The grid of a chain from its box as double-floats (lo, hi: the lowest and highest centre coordinates),
// by the rules of grid_from_bounds_s (cube cells of edge s, a multiple of 2^-10 A, from the same FP64
// formula; n_i cells with n_i s > extent_i; coarsened by 1.25 while the cells exceed the cap), with the
// FP64 pipe held to about a dozen instructions (the edge's formula): it runs in one thread on the iteration's critical
// path, where each FP64 instruction holds the sub-partition's FP64 pipe for ~84 cycles (the FP64 form
// measured 3.3 us on the 1,000-residue chain). The extents stay double-floats; n_i is the least integer
// with n_i K > 1024 extent_i (K = 1024 s), estimated in float and settled by exact comparisons (n_i K is
// an integer below 2^48, exact as a double-float). The origin is lo itself (of; ox, oy, oz are the FP64
// path's and stay 0). Returns false for a non-finite box (the grid is then one cell at the origin).
__device__ __forceinline__ bool grid_from_bounds_df(double s_base, int stencil, double cell, df lo[3], const df hi[3],
                                                    long long cap, GridInfo* out) {
    GridInfo g;
    df ext[3];
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ext[i] = sub(hi[i], lo[i]);
        finite = finite && isfinite(ext[i].hi) && isfinite(lo[i].hi);
    }
    if (!finite)
        for (int i = 0; i < 3; ++i) { lo[i] = df{0.0f, 0.0f}; ext[i] = df{0.0f, 0.0f}; }
    unsigned long long km = dfkey(ext[0]);
    km = max(km, dfkey(ext[1]));
    km = max(km, dfkey(ext[2]));
    const double emax = to_double(dfkey_inv(km));
    const double s0 = fmax(fma(1e-6, emax, s_base) * (stencil == 2 ? 0.5 : 1.0), cell);
    long long K = (long long)ceil(s0 * 1024.0);
    for (;;) {
        long long nn[3];
        bool big = false;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const df e = ldexp2(ext[i], 1024.0f);
            const float q = floorf(__fdiv_rn(e.hi, (float)K));
            if (!(q < 4194304.0f)) {  // 2^22 cells along one axis: coarsen (k K must stay below 2^48)
                big = true;
                nn[i] = 1;
                continue;
            }
            long long k = (long long)(int)q + 1;
            while (!df_gt(df_from_i64(k * K), e)) ++k;
            while (k > 1 && df_gt(df_from_i64((k - 1) * K), e)) --k;
            nn[i] = k;
        }
        if (!big && nn[0] * nn[1] * nn[2] <= cap) {
            g.nx = (int)nn[0]; g.ny = (int)nn[1]; g.nz = (int)nn[2];
            g.ncells = (int)(nn[0] * nn[1] * nn[2]);
            break;
        }
        K = (5 * K + 3) / 4;  // s <- ceil(1.25 s 1024) / 1024
    }
    g.ox = 0.0; g.oy = 0.0; g.oz = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) g.of[i] = make_float2(lo[i].hi, lo[i].lo);
    g.sf = __fdiv_rn((float)K, 1024.0f);  // exact: K < 2^24
    g.s = (double)g.sf;
    g.gpf = (float)(1e-3 + 2e-4 * g.s);
    g.inv_sf = 1.0f / g.sf;
    g.cbase = 0;
    g.pad = 0;
    *out = g;
    return finite;
}

}  // namespace dev
}  // namespace kcm
