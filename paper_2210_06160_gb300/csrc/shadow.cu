// Soft-shadow raymarch on the SDF grid (Sec. 2.4, 2.5.2, 2.5.3): one thread per
// receiver, sphere tracing toward a directional light with the triangulated
// penumbra estimate, software trilinear sampling (8 read-only loads + FP32 lerps
// in x, then y, then z; the hardware filter's fixed-point weights are avoided).
// The samples and the stop decisions use the same FP32 operations as the adjoint's
// replay; the penumbra estimate is kept as a fraction (penumbra_step).
#include "rtsdf_launch.cuh"
#include "shadow_march.cuh"

namespace rtsdf {

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Running minimum of the triangulated penumbra estimate k e / max(t - y, 1e-6)
// (Sec. 2.5.2; y = d^2 / (2 d_prev), e = sqrt(max(d^2 - y^2, 0))), held as a fraction
// rn / rd and compared by cross-multiplication, so a step takes one division (y)
// instead of two; the single division of the winning fraction comes at the end and
// reproduces its quotient.  y and the difference d^2 - y^2 (which cancels when d is
// near 2 d_prev) are the oracle's own FP32 operations; the square root after the
// cancellation is the approximate one (a few ulp, unamplified), so the visibility
// stays within a few ulp of the quotient form (it is held to 1e-4 of the oracle).
// The march's control flow depends on d alone and is unchanged.
struct Penumbra {
    float rn, rd;
};

__device__ __forceinline__ void penumbra_step(Penumbra& p, float k, float d, float d_prev, float t) {
    const float dd = d * d;
    const float y = dd / (2.0f * d_prev);
    const float a = k * sqrt_approx(fmaxf(dd - y * y, 0.0f));
    const float b = fmaxf(t - y, 1e-6f);
    if (a * p.rd < p.rn * b) {
        p.rn = a;
        p.rd = b;
    }
}

__global__ void __launch_bounds__(256) k_shadow(ShadowArgs a_in, const float* __restrict__ sdf,
                                                const float* __restrict__ pos, const float* __restrict__ nrm, int P,
                                                float* __restrict__ vis) {
    const ShadowArgs a = with_light(a_in);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float3 o = march_origin(a, pos, nrm, i);
    float t = march_start(a, i), d_prev = __int_as_float(0x7f800000);
    Penumbra pen{1.0f, 1.0f};
    bool hit = false;
    for (int s = 0; s < a.steps; ++s) {
        const float qx = o.x + t * a.L.x, qy = o.y + t * a.L.y, qz = o.z + t * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        const float d = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
        if (d <= a.hit_eps) {
            hit = true;
            break;
        }
        penumbra_step(pen, a.k, d, d_prev, t);
        d_prev = d;
        t = t + fminf(d, a.max_step);
    }
    const float res = hit ? 0.0f : pen.rn / pen.rd;
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
__global__ void __launch_bounds__(kCoherentBlock) k_shadow_coherent(ShadowArgs a_in, const float* __restrict__ sdf,
                                                                    const float* __restrict__ pos,
                                                                    const float* __restrict__ nrm, int P,
                                                                    float* __restrict__ vis,
                                                                    uint8_t* __restrict__ steps) {
    const ShadowArgs a = with_light(a_in);
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
    float tt = march_start(a, i), d_prev = __int_as_float(0x7f800000);
    Penumbra pen{1.0f, 1.0f};
    bool hit = false;
    int s = 0;
    for (; s < a.steps; ++s) {
        const float qx = o.x + tt * a.L.x, qy = o.y + tt * a.L.y, qz = o.z + tt * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        const float d = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
        if (d <= a.hit_eps) {
            hit = true;
            break;
        }
        penumbra_step(pen, a.k, d, d_prev, tt);
        d_prev = d;
        tt = tt + fminf(d, a.max_step);
    }
    const float res = hit ? 0.0f : pen.rn / pen.rd;
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
