// Soft-shadow raymarch on the SDF grid (Sec. 2.4, 2.5.2, 2.5.3): one thread per
// receiver, sphere tracing toward a directional light with the triangulated
// penumbra estimate, software trilinear sampling (8 read-only loads + FP32 lerps
// in x, then y, then z; the hardware filter's fixed-point weights are avoided).
#include "rtsdf_launch.cuh"
#include "shadow_march.cuh"

namespace rtsdf {

__global__ void __launch_bounds__(256) k_shadow(ShadowArgs a, const float* __restrict__ sdf,
                                                const float* __restrict__ pos, const float* __restrict__ nrm, int P,
                                                float* __restrict__ vis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float3 o = march_origin(a, pos, nrm, i);
    float t = march_start(a, i), res = 1.0f, d_prev = __int_as_float(0x7f800000);
    for (int s = 0; s < a.steps; ++s) {
        const float qx = o.x + t * a.L.x, qy = o.y + t * a.L.y, qz = o.z + t * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        const float d = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
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
    const ShadowArgs a = make_shadow_args(gh, p);
    if (P == 0) return RTSDF_OK;
    k_shadow<<<(P + 255) / 256, 256, 0, s>>>(a, sdf, pos, nrm, P, vis);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
