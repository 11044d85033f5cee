// C-ABI entry points of librtsdf: argument validation (before anything is
// enqueued), workspace queries, and dispatch to the kernel files.
#include <math.h>

#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

using namespace rtsdf;

namespace {

bool grid_ok(const rtsdf_grid* g) {
    if (!g) return false;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
    if (g->nx > RTSDF_MAX_DIM || g->ny > RTSDF_MAX_DIM || g->nz > RTSDF_MAX_DIM) return false;
    if (!(g->h > 0.0f) || !isfinite(g->h)) return false;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(g->origin[a])) return false;
    return true;
}

template <typename T>
bool aligned(const T* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// A device buffer argument: non-null and aligned (16 bytes for grids and
// workspaces, 4 bytes for element arrays).
template <typename T>
bool buf_ok(const T* p, size_t a) { return p != nullptr && aligned(p, a); }

bool mesh_ok(const float* verts, int32_t V, const int32_t* tris, int32_t T) {
    if (V < 0 || T < 0 || V > (1 << 28) || T > (1 << 28)) return false;
    if (T > 0 && (!buf_ok(verts, 4) || !buf_ok(tris, 4))) return false;
    if (V > 0 && !buf_ok(verts, 4)) return false;
    return true;
}

cudaStream_t cs(rtsdf_stream s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

int32_t rtsdf_version(void) { return 100; }

uint64_t rtsdf_kernel_launches(void) { return launches(); }

const char* rtsdf_status_string(rtsdf_status s) {
    switch (s) {
        case RTSDF_OK: return "ok";
        case RTSDF_EINVAL: return "invalid argument";
        case RTSDF_ENOMEM: return "workspace or buffer too small";
        case RTSDF_ECUDA: return "CUDA error";
    }
    return "unknown status";
}

size_t rtsdf_voxelize_workspace(int32_t T, const rtsdf_grid* g) {
    if (!grid_ok(g) || T < 0) return 0;
    return voxelize_workspace(T, *g);
}

rtsdf_status rtsdf_voxelize(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid* g,
                            int32_t* seed, int32_t* rep_tri, void* ws, size_t ws_bytes, rtsdf_counters* counters,
                            rtsdf_stream stream) {
    if (!grid_ok(g) || !mesh_ok(verts, V, tris, T)) return RTSDF_EINVAL;
    if (!buf_ok(seed, 16) || !buf_ok(rep_tri, 16) || !buf_ok(ws, 256)) return RTSDF_EINVAL;
    if (counters && !aligned(counters, 8)) return RTSDF_EINVAL;
    if (ws_bytes < voxelize_workspace(T, *g)) return RTSDF_ENOMEM;
    return voxelize(verts, V, tris, T, *g, seed, rep_tri, ws, counters, cs(stream));
}

size_t rtsdf_bvh_bytes(int32_t T) { return T < 0 ? 0 : bvh_bytes(T); }
size_t rtsdf_bvh_workspace(int32_t T) { return T < 0 ? 0 : bvh_workspace(T); }

rtsdf_status rtsdf_build_bvh(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid* g,
                             void* bvh, size_t bvh_bytes_, void* ws, size_t ws_bytes, rtsdf_counters* counters,
                             rtsdf_stream stream) {
    if (!grid_ok(g) || !mesh_ok(verts, V, tris, T)) return RTSDF_EINVAL;
    if (!buf_ok(bvh, 256) || !buf_ok(ws, 256)) return RTSDF_EINVAL;
    if (counters && !aligned(counters, 8)) return RTSDF_EINVAL;
    if (bvh_bytes_ < bvh_bytes(T) || ws_bytes < bvh_workspace(T)) return RTSDF_ENOMEM;
    return build_bvh(verts, V, tris, T, *g, bvh, ws, counters, cs(stream));
}

rtsdf_status rtsdf_jfa(const rtsdf_grid* g, int32_t* buf_a, int32_t* buf_b, const int32_t* steps, int32_t nsteps,
                       int32_t** result, rtsdf_stream stream) {
    if (!grid_ok(g) || !buf_ok(buf_a, 16) || !buf_ok(buf_b, 16) || buf_a == buf_b || !result) return RTSDF_EINVAL;
    if (nsteps < 0 || (nsteps > 0 && !steps)) return RTSDF_EINVAL;
    for (int32_t i = 0; i < nsteps; ++i)
        if (steps[i] < 1 || steps[i] > RTSDF_MAX_DIM) return RTSDF_EINVAL;
    return jfa(*g, buf_a, buf_b, steps, nsteps, result, cs(stream));
}

size_t rtsdf_refine_workspace(const rtsdf_grid* g) { return grid_ok(g) ? refine_workspace(*g) : 0; }

namespace {

// The coarse grid of a two-resolution call: same origin, an edge of `ratio` fine
// edges (ratio a positive integer, to 1e-6 relative), dims = ceil(fine dims / ratio).
int coarse_ratio(const rtsdf_grid* fine, const rtsdf_grid* coarse) {
    if (!grid_ok(coarse)) return 0;
    for (int a = 0; a < 3; ++a)
        if (coarse->origin[a] != fine->origin[a]) return 0;
    const double r = (double)coarse->h / (double)fine->h;
    const int ri = (int)(r + 0.5);
    if (ri < 1 || ri > 64 || fabs(r - ri) > 1e-6 * r) return 0;
    if (coarse->nx != (fine->nx + ri - 1) / ri || coarse->ny != (fine->ny + ri - 1) / ri ||
        coarse->nz != (fine->nz + ri - 1) / ri)
        return 0;
    return ri;
}

rtsdf_status refine_checked(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                            const void* bvh, size_t bvh_bytes_, const int32_t* nearest, const int32_t* rep_tri,
                            const rtsdf_refine_params* p, uint32_t* dist_bits, uint32_t* front, uint32_t* back,
                            float* sdf_out, uint32_t* win_ray, int32_t* win_tri, void* ws, size_t ws_bytes,
                            rtsdf_counters* counters, rtsdf_stream stream, const rtsdf_grid* coarse = nullptr) {
    int ratio = 1;
    if (coarse) {
        if (!grid_ok(g)) return RTSDF_EINVAL;
        ratio = coarse_ratio(g, coarse);
        if (ratio == 0) return RTSDF_EINVAL;
    }
    if (!grid_ok(g) || !mesh_ok(verts, V, tris, T) || !p) return RTSDF_EINVAL;
    if (!buf_ok(bvh, 256) || !buf_ok(nearest, 16) || !buf_ok(rep_tri, 16) || !buf_ok(dist_bits, 16) ||
        !buf_ok(front, 16) || !buf_ok(back, 16) || !buf_ok(sdf_out, 16) || !buf_ok(ws, 256))
        return RTSDF_EINVAL;
    if (counters && !aligned(counters, 8)) return RTSDF_EINVAL;
    if (p->rays_per_voxel < 1 || p->rays_per_voxel > 4096) return RTSDF_EINVAL;
    if (p->accumulate < 0 || p->accumulate > 2) return RTSDF_EINVAL;
    if (p->accumulate == 2 && !(p->decay_alpha >= 0.0f && p->decay_alpha <= 1.0f)) return RTSDF_EINVAL;
    if (!(p->mask_vox >= 0.0f) || !isfinite(p->mask_vox) || !(p->max_ray_vox > 0.0f) || !isfinite(p->beta_vox))
        return RTSDF_EINVAL;
    if (bvh_bytes_ < bvh_bytes(T)) return RTSDF_ENOMEM;
    if (ws_bytes < refine_workspace(*g)) return RTSDF_ENOMEM;
    return refine(*g, T, bvh, nearest, rep_tri, *p, dist_bits, front, back, sdf_out, ws, counters,
                  win_ray, win_tri, coarse, ratio, cs(stream));
}

bool refine_params_ok(const rtsdf_refine_params* p) {
    return p && p->rays_per_voxel >= 1 && p->rays_per_voxel <= 4096 && p->mask_vox >= 0.0f &&
           isfinite(p->mask_vox) && isfinite(p->beta_vox);
}

bool shadow_params_ok(const rtsdf_shadow_params* p) {
    if (!p) return false;
    bool light_ok;
    if (p->light_dir_device) {
        light_ok = reinterpret_cast<uintptr_t>(p->light_dir_device) % 4 == 0;  // read on the device
    } else {
        const float* l = p->light_dir;
        const float len2 = l[0] * l[0] + l[1] * l[1] + l[2] * l[2];
        light_ok = len2 > 0.0f && isfinite(len2);
    }
    return light_ok && p->steps >= 0 && p->max_step_vox > 0.0f && isfinite(p->k) && p->jitter_vox >= 0.0f &&
           isfinite(p->jitter_vox);
}

}  // namespace

rtsdf_status rtsdf_refine(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                          const void* bvh, size_t bvh_bytes_, const int32_t* nearest, const int32_t* rep_tri,
                          const rtsdf_refine_params* p, uint32_t* dist_bits, uint32_t* front, uint32_t* back,
                          float* sdf_out, void* ws, size_t ws_bytes, rtsdf_counters* counters, rtsdf_stream stream) {
    return refine_checked(g, verts, V, tris, T, bvh, bvh_bytes_, nearest, rep_tri, p, dist_bits, front, back, sdf_out,
                          nullptr, nullptr, ws, ws_bytes, counters, stream);
}

rtsdf_status rtsdf_refine_tracked(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                                  const void* bvh, size_t bvh_bytes_, const int32_t* nearest, const int32_t* rep_tri,
                                  const rtsdf_refine_params* p, uint32_t* dist_bits, uint32_t* front, uint32_t* back,
                                  float* sdf_out, uint32_t* win_ray, int32_t* win_tri, void* ws, size_t ws_bytes,
                                  rtsdf_counters* counters, rtsdf_stream stream) {
    if (!buf_ok(win_ray, 16) || !buf_ok(win_tri, 16)) return RTSDF_EINVAL;
    return refine_checked(g, verts, V, tris, T, bvh, bvh_bytes_, nearest, rep_tri, p, dist_bits, front, back, sdf_out,
                          win_ray, win_tri, ws, ws_bytes, counters, stream);
}

rtsdf_status rtsdf_refine_2res(const rtsdf_grid* fine, const rtsdf_grid* coarse, const float* verts, int32_t V,
                               const int32_t* tris, int32_t T, const void* bvh, size_t bvh_bytes_,
                               const int32_t* nearest, const int32_t* rep_tri, const rtsdf_refine_params* p,
                               uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf_out, void* ws,
                               size_t ws_bytes, rtsdf_counters* counters, rtsdf_stream stream) {
    if (!coarse) return RTSDF_EINVAL;
    return refine_checked(fine, verts, V, tris, T, bvh, bvh_bytes_, nearest, rep_tri, p, dist_bits, front, back,
                          sdf_out, nullptr, nullptr, ws, ws_bytes, counters, stream, coarse);
}

rtsdf_status rtsdf_shadow(const rtsdf_grid* g, const float* sdf, const float* pos, const float* nrm, int32_t P,
                          const rtsdf_shadow_params* p, float* vis, rtsdf_stream stream) {
    if (!grid_ok(g) || !p || P < 0 || !buf_ok(sdf, 16)) return RTSDF_EINVAL;
    if (P > 0 && (!buf_ok(pos, 4) || !buf_ok(nrm, 4) || !buf_ok(vis, 4))) return RTSDF_EINVAL;
    if (!shadow_params_ok(p)) return RTSDF_EINVAL;
    return shadow(*g, sdf, pos, nrm, P, *p, vis, cs(stream));
}

rtsdf_status rtsdf_shadow_coherent(const rtsdf_grid* g, const float* sdf, const float* pos, const float* nrm,
                                   int32_t P, const rtsdf_shadow_params* p, float* vis, uint8_t* steps,
                                   rtsdf_stream stream) {
    if (!grid_ok(g) || !p || P < 0 || !buf_ok(sdf, 16)) return RTSDF_EINVAL;
    if (P > 0 && (!buf_ok(pos, 4) || !buf_ok(nrm, 4) || !buf_ok(vis, 4) || !steps)) return RTSDF_EINVAL;
    if (!shadow_params_ok(p)) return RTSDF_EINVAL;
    return shadow_coherent(*g, sdf, pos, nrm, P, *p, vis, steps, cs(stream));
}

rtsdf_status rtsdf_sample(const rtsdf_grid* g, const float* sdf, const float* pts, int32_t M, float* out,
                          rtsdf_stream stream) {
    if (!grid_ok(g) || M < 0 || !buf_ok(sdf, 16)) return RTSDF_EINVAL;
    if (M > 0 && (!buf_ok(pts, 4) || !buf_ok(out, 4))) return RTSDF_EINVAL;
    return sample(*g, sdf, pts, M, out, cs(stream));
}

size_t rtsdf_backward_workspace(const rtsdf_grid* g) { return grid_ok(g) ? backward_workspace(*g) : 0; }

rtsdf_status rtsdf_backward(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                            const int32_t* nearest, const int32_t* rep_tri, const uint32_t* front,
                            const uint32_t* back, const uint32_t* win_ray, const int32_t* win_tri,
                            const rtsdf_refine_params* rp, const float* sdf, const float* pts, int32_t M,
                            const float* d_samples, const float* pos, const float* nrm, int32_t P,
                            const rtsdf_shadow_params* sp, const float* d_vis, float* d_verts, float* d_light,
                            void* ws, size_t ws_bytes, rtsdf_stream stream) {
    if (!grid_ok(g) || !mesh_ok(verts, V, tris, T) || !refine_params_ok(rp) || !shadow_params_ok(sp))
        return RTSDF_EINVAL;
    if (sp->steps > RTSDF_BACKWARD_MAX_STEPS || M < 0 || P < 0) return RTSDF_EINVAL;
    if (!buf_ok(nearest, 16) || !buf_ok(rep_tri, 16) || !buf_ok(front, 16) || !buf_ok(back, 16) ||
        !buf_ok(win_ray, 16) || !buf_ok(win_tri, 16) || !buf_ok(sdf, 16) || !buf_ok(d_light, 4) ||
        !buf_ok(ws, 256))
        return RTSDF_EINVAL;
    if (V > 0 && !buf_ok(d_verts, 4)) return RTSDF_EINVAL;
    if (M > 0 && (!buf_ok(pts, 4) || !buf_ok(d_samples, 4))) return RTSDF_EINVAL;
    if (P > 0 && (!buf_ok(pos, 4) || !buf_ok(nrm, 4) || !buf_ok(d_vis, 4))) return RTSDF_EINVAL;
    if (ws_bytes < backward_workspace(*g)) return RTSDF_ENOMEM;
    return backward(*g, verts, V, tris, T, nearest, rep_tri, front, back, win_ray, win_tri, *rp, sdf, pts, M,
                    d_samples, pos, nrm, P, *sp, d_vis, d_verts, d_light, ws, cs(stream));
}

}  // extern "C"
