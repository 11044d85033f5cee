// The pieces of the soft-shadow raymarch (Sec. 2.4, 2.5.2, 2.5.3) that its forward
// kernel and its adjoint share, so the adjoint replays exactly the forward's FP32
// march: the launch arguments, the software trilinear sample and the ray origin.
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

struct ShadowArgs {
    GridD g;
    float3 L;  // unit direction toward the light (FP32, normalised on the host)
    const float* Ldev;  // the caller's device light vector, or null (then L holds the direction)
    float k;
    int steps;
    float max_step, start_off, normal_off, hit_eps, bias;
    float jitter;
    uint32_t frame;
};

inline ShadowArgs make_shadow_args(const rtsdf_grid& gh, const rtsdf_shadow_params& p) {
    ShadowArgs a;
    a.g = to_dev(gh);
    a.Ldev = p.light_dir_device;
    if (a.Ldev) {
        a.L = make_float3(0.0f, 0.0f, 0.0f);  // resolved on the device (with_light)
    } else {
        const float* l = p.light_dir;
        const float len = sqrtf(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
        a.L = make_float3(l[0] / len, l[1] / len, l[2] / len);
    }
    a.k = p.k;
    a.steps = p.steps;
    a.max_step = p.max_step_vox;
    a.start_off = p.start_offset_vox;
    a.normal_off = p.normal_offset_vox;
    a.hit_eps = p.hit_eps_vox;
    a.bias = p.bias_vox;
    a.jitter = p.jitter_vox;
    a.frame = p.frame_index;
    return a;
}

// Length of a light vector and its unit direction: the squared length summed x, y,
// z, a correctly rounded square root and three correctly rounded divisions, the
// same FP32 operations on the host (make_shadow_args) and on the device.
__device__ __forceinline__ float3 unit_light(const float* __restrict__ l, float& len) {
    const float l0 = __ldg(l), l1 = __ldg(l + 1), l2 = __ldg(l + 2);
    len = sqrtf(l0 * l0 + l1 * l1 + l2 * l2);
    return make_float3(l0 / len, l1 / len, l2 / len);
}

// The launch's arguments with the light direction resolved: from the caller's device
// vector when one is given, else as normalised on the host.
__device__ __forceinline__ ShadowArgs with_light(const ShadowArgs& a) {
    ShadowArgs r = a;
    if (a.Ldev) {
        float len;
        r.L = unit_light(a.Ldev, len);
    }
    return r;
}

// First sample distance of receiver i: start_off, moved along the light by a
// per-receiver, per-frame jitter (Sec. 2.5.2) drawn from Philox4x32-10.
__device__ __forceinline__ float march_start(const ShadowArgs& a, int i) {
    if (a.jitter == 0.0f) return a.start_off;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)i, a.frame, 0x4A177E2u, 0u), 0x51AD0u, 0x7E2u);
    const float u = (float)(x.x >> 8) * 0x1p-24f;
    return a.start_off + a.jitter * u;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return a + (b - a) * t; }

// Cell of a trilinear sample at voxel coordinate q (voxel centres at i + 0.5,
// clamp to edge): the 8 corner offsets (x fastest: 000,100,010,110,001,101,011,111)
// and the fractional position.
struct Cell {
    int32_t c[8];
    float fx, fy, fz;
};

__device__ __forceinline__ Cell cell_at(const GridD& g, float qx, float qy, float qz) {
    const float sx = qx - 0.5f, sy = qy - 0.5f, sz = qz - 0.5f;
    const float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
    Cell c;
    c.fx = sx - flx;
    c.fy = sy - fly;
    c.fz = sz - flz;
    const int ix = (int)flx, iy = (int)fly, iz = (int)flz;
    const int x0 = min(max(ix, 0), g.nx - 1), x1 = min(max(ix + 1, 0), g.nx - 1);
    const int y0 = min(max(iy, 0), g.ny - 1), y1 = min(max(iy + 1, 0), g.ny - 1);
    const int z0 = min(max(iz, 0), g.nz - 1), z1 = min(max(iz + 1, 0), g.nz - 1);
    const int32_t p = g.nx * g.ny;  // grids have at most 1023^3 < 2^31 voxels
    const int32_t r00 = z0 * p + y0 * g.nx, r10 = z0 * p + y1 * g.nx;
    const int32_t r01 = z1 * p + y0 * g.nx, r11 = z1 * p + y1 * g.nx;
    c.c[0] = r00 + x0; c.c[1] = r00 + x1; c.c[2] = r10 + x0; c.c[3] = r10 + x1;
    c.c[4] = r01 + x0; c.c[5] = r01 + x1; c.c[6] = r11 + x0; c.c[7] = r11 + x1;
    return c;
}

// FP32 lerps in x, then y, then z.
__device__ __forceinline__ float cell_value(const float v[8], const Cell& c) {
    const float c00 = lerpf(v[0], v[1], c.fx), c10 = lerpf(v[2], v[3], c.fx);
    const float c01 = lerpf(v[4], v[5], c.fx), c11 = lerpf(v[6], v[7], c.fx);
    return lerpf(lerpf(c00, c10, c.fy), lerpf(c01, c11, c.fy), c.fz);
}

__device__ __forceinline__ void cell_load(const float* __restrict__ f, const Cell& c, float v[8]) {
#pragma unroll
    for (int b = 0; b < 8; ++b) v[b] = __ldg(f + c.c[b]);
}

__device__ __forceinline__ float trilinear(const float* __restrict__ f, const GridD& g, float qx, float qy, float qz) {
    const Cell c = cell_at(g, qx, qy, qz);
    float v[8];
    cell_load(f, c, v);
    return cell_value(v, c);
}

// Ray origin of receiver i in voxel coordinates: its position lifted by
// normal_off voxels along its normal (Sec. 2.5.3).
__device__ __forceinline__ float3 march_origin(const ShadowArgs& a, const float* __restrict__ pos,
                                               const float* __restrict__ nrm, int i) {
    const GridD& g = a.g;
    const float px = __ldg(pos + 3 * (int64_t)i), py = __ldg(pos + 3 * (int64_t)i + 1),
                pz = __ldg(pos + 3 * (int64_t)i + 2);
    const float nx = __ldg(nrm + 3 * (int64_t)i), ny = __ldg(nrm + 3 * (int64_t)i + 1),
                nz = __ldg(nrm + 3 * (int64_t)i + 2);
    return make_float3((px - g.ox) / g.h + a.normal_off * nx, (py - g.oy) / g.h + a.normal_off * ny,
                       (pz - g.oz) / g.h + a.normal_off * nz);
}

__device__ __forceinline__ bool outside_box(const GridD& g, float qx, float qy, float qz) {
    return qx < 0.0f || qx > (float)g.nx || qy < 0.0f || qy > (float)g.ny || qz < 0.0f || qz > (float)g.nz;
}

}  // namespace rtsdf
