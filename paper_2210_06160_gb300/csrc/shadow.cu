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

constexpr int kCoherentBlock = 512;  // receivers regrouped per block

// The march of k_shadow with the lanes regrouped: each block of kCoherentBlock
// consecutive receivers first sorts them by the march length they had in the previous
// call (a counting sort in shared memory), so that the lanes of a warp take receivers
// that march about as long and fewer lanes idle while the longest march of the warp
// runs on.  Each receiver's march is independent of the others, so the outputs are
// those of k_shadow; steps[i] receives the new length (the step at which the march
// stopped, at most 255).
__global__ void __launch_bounds__(kCoherentBlock) k_shadow_coherent(ShadowArgs a, const float* __restrict__ sdf,
                                                                    const float* __restrict__ pos,
                                                                    const float* __restrict__ nrm, int P,
                                                                    float* __restrict__ vis,
                                                                    uint8_t* __restrict__ steps) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t wsum[8];
    __shared__ uint16_t perm[kCoherentBlock];
    const int t = threadIdx.x, lane = t & 31;
    const int base = blockIdx.x * kCoherentBlock;
    const int n = min(kCoherentBlock, P - base);
    if (t < 256) hist[t] = 0u;
    __syncthreads();
    uint32_t len = 0u, rank = 0u;
    if (t < n) {
        len = steps[base + t];
        rank = atomicAdd(&hist[len], 1u);
    }
    __syncthreads();
    // exclusive scan of the 256 bins: eight warps scan 32 bins each, then add the
    // totals of the warps before theirs
    uint32_t cnt = 0u, incl = 0u;
    if (t < 256) {
        cnt = incl = hist[t];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[t >> 5] = incl;
    }
    __syncthreads();
    if (t < 256) {
        uint32_t before = 0u;
        for (int w = 0; w < (t >> 5); ++w) before += wsum[w];
        hist[t] = before + incl - cnt;
    }
    __syncthreads();
    if (t < n) perm[hist[len] + rank] = (uint16_t)t;
    __syncthreads();
    if (t >= n) return;
    const int i = base + perm[t];
    const float3 o = march_origin(a, pos, nrm, i);
    float tt = march_start(a, i), res = 1.0f, d_prev = __int_as_float(0x7f800000);
    int s = 0;
    for (; s < a.steps; ++s) {
        const float qx = o.x + tt * a.L.x, qy = o.y + tt * a.L.y, qz = o.z + tt * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        const float d = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
        if (d <= a.hit_eps) {
            res = 0.0f;
            break;
        }
        const float dd = d * d;
        const float y = dd / (2.0f * d_prev);
        const float e = sqrtf(fmaxf(dd - y * y, 0.0f));
        res = fminf(res, (a.k * e) / fmaxf(tt - y, 1e-6f));
        d_prev = d;
        tt = tt + fminf(d, a.max_step);
    }
    vis[i] = fminf(fmaxf(res, 0.0f), 1.0f);
    steps[i] = (uint8_t)min(s, 255);
}

rtsdf_status shadow_coherent(const rtsdf_grid& gh, const float* sdf, const float* pos, const float* nrm, int32_t P,
                             const rtsdf_shadow_params& p, float* vis, uint8_t* steps, cudaStream_t s) {
    const ShadowArgs a = make_shadow_args(gh, p);
    if (P == 0) return RTSDF_OK;
    k_shadow_coherent<<<(P + kCoherentBlock - 1) / kCoherentBlock, kCoherentBlock, 0, s>>>(a, sdf, pos, nrm, P, vis,
                                                                                          steps);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
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
