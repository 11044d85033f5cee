// Soft-shadow raymarch on the SDF grid (Sec. 2.4, 2.5.2, 2.5.3): one thread per
// receiver, sphere tracing toward a directional light with the triangulated
// penumbra estimate, software trilinear sampling (8 read-only loads + FP32 lerps
// in x, then y, then z; the hardware filter's fixed-point weights are avoided).
#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

struct ShadowArgs {
    GridD g;
    float3 L;
    float k;
    int steps;
    float max_step, start_off, normal_off, hit_eps, bias;
};

__device__ __forceinline__ float lerpf(float a, float b, float t) { return a + (b - a) * t; }

__device__ __forceinline__ float trilinear(const float* __restrict__ f, const GridD& g, float qx, float qy, float qz) {
    const float sx = qx - 0.5f, sy = qy - 0.5f, sz = qz - 0.5f;
    const float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
    const float fx = sx - flx, fy = sy - fly, fz = sz - flz;
    const int ix = (int)flx, iy = (int)fly, iz = (int)flz;
    const int x0 = min(max(ix, 0), g.nx - 1), x1 = min(max(ix + 1, 0), g.nx - 1);
    const int y0 = min(max(iy, 0), g.ny - 1), y1 = min(max(iy + 1, 0), g.ny - 1);
    const int z0 = min(max(iz, 0), g.nz - 1), z1 = min(max(iz + 1, 0), g.nz - 1);
    const int64_t p = (int64_t)g.nx * g.ny;
    const float* r00 = f + z0 * p + (int64_t)y0 * g.nx;
    const float* r10 = f + z0 * p + (int64_t)y1 * g.nx;
    const float* r01 = f + z1 * p + (int64_t)y0 * g.nx;
    const float* r11 = f + z1 * p + (int64_t)y1 * g.nx;
    const float c00 = lerpf(__ldg(r00 + x0), __ldg(r00 + x1), fx);
    const float c10 = lerpf(__ldg(r10 + x0), __ldg(r10 + x1), fx);
    const float c01 = lerpf(__ldg(r01 + x0), __ldg(r01 + x1), fx);
    const float c11 = lerpf(__ldg(r11 + x0), __ldg(r11 + x1), fx);
    return lerpf(lerpf(c00, c10, fy), lerpf(c01, c11, fy), fz);
}

__global__ void __launch_bounds__(256) k_shadow(ShadowArgs a, const float* __restrict__ sdf,
                                                const float* __restrict__ pos, const float* __restrict__ nrm, int P,
                                                float* __restrict__ vis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const GridD& g = a.g;
    const float px = __ldg(pos + 3 * (int64_t)i), py = __ldg(pos + 3 * (int64_t)i + 1), pz = __ldg(pos + 3 * (int64_t)i + 2);
    const float nx = __ldg(nrm + 3 * (int64_t)i), ny = __ldg(nrm + 3 * (int64_t)i + 1), nz = __ldg(nrm + 3 * (int64_t)i + 2);
    const float ox = (px - g.ox) / g.h + a.normal_off * nx;
    const float oy = (py - g.oy) / g.h + a.normal_off * ny;
    const float oz = (pz - g.oz) / g.h + a.normal_off * nz;
    const float gx = (float)g.nx, gy = (float)g.ny, gz = (float)g.nz;
    float t = a.start_off, res = 1.0f, d_prev = __int_as_float(0x7f800000);
    for (int s = 0; s < a.steps; ++s) {
        const float qx = ox + t * a.L.x, qy = oy + t * a.L.y, qz = oz + t * a.L.z;
        if (qx < 0.0f || qx > gx || qy < 0.0f || qy > gy || qz < 0.0f || qz > gz) break;
        const float d = trilinear(sdf, g, qx, qy, qz) - a.bias;
        if (d <= a.hit_eps) {
            res = 0.0f;
            break;
        }
        const float dd = d * d;
        const float y = dd / (2.0f * d_prev);
        const float e = sqrtf(fmaxf(dd - y * y, 0.0f));
        res = fminf(res, (a.k * e) / fmaxf(t - y, 1e-6f));
        d_prev = d;
        t = t + fminf(d, a.max_step);
    }
    vis[i] = fminf(fmaxf(res, 0.0f), 1.0f);
}

rtsdf_status shadow(const rtsdf_grid& gh, const float* sdf, const float* pos, const float* nrm, int32_t P,
                    const rtsdf_shadow_params& p, float* vis, cudaStream_t s) {
    ShadowArgs a;
    a.g = to_dev(gh);
    const float* l = p.light_dir;
    const float len = sqrtf(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    a.L = make_float3(l[0] / len, l[1] / len, l[2] / len);
    a.k = p.k;
    a.steps = p.steps;
    a.max_step = p.max_step_vox;
    a.start_off = p.start_offset_vox;
    a.normal_off = p.normal_offset_vox;
    a.hit_eps = p.hit_eps_vox;
    a.bias = p.bias_vox;
    if (P == 0) return RTSDF_OK;
    k_shadow<<<(P + 255) / 256, 256, 0, s>>>(a, sdf, pos, nrm, P, vis);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
