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

}  // namespace dev
}  // namespace kcm
