// The soft-shadow raymarch with the field read through a 3D texture: hardware
// trilinear filtering (Sec. 2.1: a uniform grid stored as a 3D texture allows
// hardware interpolation).  Same march as k_shadow; only the sample differs: the
// texture unit's linear filter (fixed-point weights with 8 fractional bits) instead
// of the software FP32 lerps, so results differ from the FP32 path by a fraction of
// a texel in distance (tolerance documented with rtsdf_shadow_tex).
#include <new>

#include "rtsdf_launch.cuh"
#include "shadow_march.cuh"

struct rtsdf_texture {
    cudaArray_t array = nullptr;
    cudaTextureObject_t tex = 0;
    rtsdf_grid grid{};
};

namespace rtsdf {

__global__ void __launch_bounds__(256) k_shadow_tex(ShadowArgs a_in, cudaTextureObject_t tex,
                                                    const float* __restrict__ pos, const float* __restrict__ nrm,
                                                    int P, float* __restrict__ vis) {
    const ShadowArgs a = with_light(a_in);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float3 o = march_origin(a, pos, nrm, i);
    float t = march_start(a, i), res = 1.0f, d_prev = __int_as_float(0x7f800000);
    for (int s = 0; s < a.steps; ++s) {
        const float qx = o.x + t * a.L.x, qy = o.y + t * a.L.y, qz = o.z + t * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        // unnormalised coordinates: texel centres at i + 0.5, the grid's convention
        const float d = tex3D<float>(tex, qx, qy, qz) - a.bias;
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

}  // namespace rtsdf

using namespace rtsdf;

extern "C" {

rtsdf_status rtsdf_texture_create(const rtsdf_grid* g, rtsdf_texture** out) {
    if (!out) return RTSDF_EINVAL;
    *out = nullptr;
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > RTSDF_MAX_DIM || g->ny > RTSDF_MAX_DIM ||
        g->nz > RTSDF_MAX_DIM || !(g->h > 0.0f))
        return RTSDF_EINVAL;
    rtsdf_texture* t = new (std::nothrow) rtsdf_texture();
    if (!t) return RTSDF_ENOMEM;
    t->grid = *g;
    const cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
    if (cudaMalloc3DArray(&t->array, &ch, make_cudaExtent(g->nx, g->ny, g->nz), 0) != cudaSuccess) {
        delete t;
        return RTSDF_ECUDA;
    }
    cudaResourceDesc res{};
    res.resType = cudaResourceTypeArray;
    res.res.array.array = t->array;
    cudaTextureDesc td{};
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    if (cudaCreateTextureObject(&t->tex, &res, &td, nullptr) != cudaSuccess) {
        cudaFreeArray(t->array);
        delete t;
        return RTSDF_ECUDA;
    }
    *out = t;
    return RTSDF_OK;
}

void rtsdf_texture_destroy(rtsdf_texture* t) {
    if (!t) return;
    if (t->tex) cudaDestroyTextureObject(t->tex);
    if (t->array) cudaFreeArray(t->array);
    delete t;
}

rtsdf_status rtsdf_texture_upload(rtsdf_texture* t, const float* sdf, rtsdf_stream stream) {
    if (!t || !sdf || reinterpret_cast<uintptr_t>(sdf) % 16) return RTSDF_EINVAL;
    const rtsdf_grid& g = t->grid;
    cudaMemcpy3DParms p{};
    p.srcPtr = make_cudaPitchedPtr(const_cast<float*>(sdf), sizeof(float) * (size_t)g.nx, (size_t)g.nx, (size_t)g.ny);
    p.dstArray = t->array;
    p.extent = make_cudaExtent(g.nx, g.ny, g.nz);
    p.kind = cudaMemcpyDeviceToDevice;
    RTSDF_CUDA(cudaMemcpy3DAsync(&p, reinterpret_cast<cudaStream_t>(stream)));
    return RTSDF_OK;
}

rtsdf_status rtsdf_shadow_tex(const rtsdf_texture* t, const float* pos, const float* nrm, int32_t P,
                              const rtsdf_shadow_params* p, float* vis, rtsdf_stream stream) {
    if (!t || !p || P < 0) return RTSDF_EINVAL;
    if (P > 0 && (!pos || !nrm || !vis || reinterpret_cast<uintptr_t>(pos) % 4 ||
                  reinterpret_cast<uintptr_t>(nrm) % 4 || reinterpret_cast<uintptr_t>(vis) % 4))
        return RTSDF_EINVAL;
    const float* l = p->light_dir;
    const float len2 = l[0] * l[0] + l[1] * l[1] + l[2] * l[2];
    const bool light_ok = p->light_dir_device ? reinterpret_cast<uintptr_t>(p->light_dir_device) % 4 == 0
                                              : len2 > 0.0f;
    if (!light_ok || p->steps < 0 || !(p->max_step_vox > 0.0f) || !(p->jitter_vox >= 0.0f)) return RTSDF_EINVAL;
    const ShadowArgs a = make_shadow_args(t->grid, *p);
    if (P == 0) return RTSDF_OK;
    k_shadow_tex<<<(P + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a, t->tex, pos, nrm, P, vis);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // extern "C"
