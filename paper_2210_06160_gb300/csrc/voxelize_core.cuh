// Voxel ranges of triangles for the conservative voxelizer (Sec. 2.2), shared by
// the single-scene (voxelize.cu) and batched (batch.cu) kernels.
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

constexpr int kBrick = 8;

// Voxel range of a triangle along one axis: the closed triangle can touch voxel i
// (spanning [i, i+1]) only if min <= i + 1 and max >= i.
__device__ __forceinline__ bool axis_range(float a, float b, float c, int n, int& lo, int& hi) {
    const float mn = fminf(fminf(a, b), c), mx = fmaxf(fmaxf(a, b), c);
    const float l = fmaxf(ceilf(mn) - 1.0f, 0.0f);
    const float h = fminf(floorf(mx), (float)n - 1.0f);
    if (!(l <= h)) return false;
    lo = (int)l;
    hi = (int)h;
    return true;
}

struct TriRange {
    int lo[3], hi[3];
};

__device__ __forceinline__ bool tri_range(float3 a, float3 b, float3 c, const GridD& g, TriRange& r) {
    return axis_range(a.x, b.x, c.x, g.nx, r.lo[0], r.hi[0]) && axis_range(a.y, b.y, c.y, g.ny, r.lo[1], r.hi[1]) &&
           axis_range(a.z, b.z, c.z, g.nz, r.lo[2], r.hi[2]);
}

// Bricks of a triangle's voxel range.
__device__ __forceinline__ uint32_t range_bricks(const TriRange& r) {
    return (uint32_t)((r.hi[0] / kBrick - r.lo[0] / kBrick + 1) * (r.hi[1] / kBrick - r.lo[1] / kBrick + 1) *
                      (r.hi[2] / kBrick - r.lo[2] / kBrick + 1));
}

// The voxel tests of one (triangle, brick) item: a warp culls the brick (enlarged
// by a margin far above FP32 rounding of the voxel test), then its lanes test the
// voxels of brick ∩ range and lower each overlapped voxel's 64-bit key
// (closest-point distance^2 bits, triangle id) with atomicMin.
__device__ __forceinline__ void vox_item(float3 a, float3 b, float3 c, const TriRange& r, int local, int tri_id,
                                         const GridD& g, unsigned long long* __restrict__ keys) {
    const uint32_t lane = lane_id();
    const int nbx = r.hi[0] / kBrick - r.lo[0] / kBrick + 1;
    const int nby = r.hi[1] / kBrick - r.lo[1] / kBrick + 1;
    const int bx = r.lo[0] / kBrick + local % nbx;
    const int by = r.lo[1] / kBrick + (local / nbx) % nby;
    const int bz = r.lo[2] / kBrick + local / (nbx * nby);
    const float3 bc = make_float3((float)(bx * kBrick) + 0.5f * kBrick, (float)(by * kBrick) + 0.5f * kBrick,
                                  (float)(bz * kBrick) + 0.5f * kBrick);
    if (!tri_box_overlap(a, b, c, bc, 0.5f * kBrick + 0.0625f)) return;
    const int x0 = max(r.lo[0], bx * kBrick), x1 = min(r.hi[0], bx * kBrick + kBrick - 1);
    const int y0 = max(r.lo[1], by * kBrick), y1 = min(r.hi[1], by * kBrick + kBrick - 1);
    const int z0 = max(r.lo[2], bz * kBrick), z1 = min(r.hi[2], bz * kBrick + kBrick - 1);
    const int sx = x1 - x0 + 1, sy = y1 - y0 + 1, nsub = sx * sy * (z1 - z0 + 1);
    for (int v = (int)lane; v < nsub; v += kWarp) {
        const int i = x0 + v % sx, j = y0 + (v / sx) % sy, k = z0 + v / (sx * sy);
        const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
        if (!tri_box_overlap(a, b, c, p, 0.5f)) continue;
        const float d2 = closest_d2(p, a, b, c);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned long long)(uint32_t)tri_id;
        const int64_t lin = ((int64_t)k * g.ny + j) * g.nx + i;
        atomicMin(keys + lin, key);
    }
}

}  // namespace rtsdf
