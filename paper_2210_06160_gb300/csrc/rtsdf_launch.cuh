// Host-side helpers shared by the kernel files: error macros, device properties,
// the device-wide scan, and the per-step entry points the C-ABI layer calls.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rtsdf.h"

#define RTSDF_CUDA(expr)                                  \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return RTSDF_ECUDA;        \
    } while (0)

// Checks the launch just enqueued and counts it.
#define RTSDF_LAUNCHED()                                  \
    do {                                                  \
        RTSDF_CUDA(cudaGetLastError());                   \
        ::rtsdf::note_launch();                           \
    } while (0)

#define RTSDF_TRY(expr)                                   \
    do {                                                  \
        rtsdf_status s_ = (expr);                         \
        if (s_ != RTSDF_OK) return s_;                    \
    } while (0)

namespace rtsdf {

// Counts one enqueued kernel (see rtsdf_kernel_launches).
void note_launch(int n = 1);
uint64_t launches();

// SM count of the current device (cached per device).
int num_sms();

// Exclusive scan of n uint32 counts into n+1 uint64 offsets (out[n] = total).
size_t scan_u32_to_u64_scratch(size_t n);
rtsdf_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, size_t n, void* scratch, cudaStream_t s);

// Steps (one per kernel file).  Arguments are validated by the C-ABI layer.
size_t voxelize_workspace(int32_t T, const rtsdf_grid& g);
rtsdf_status voxelize(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid& g,
                      int32_t* seed, int32_t* rep_tri, void* ws, rtsdf_counters* counters, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs over the low key_bits bits, 8 bits
// per pass, ping-ponging between (ka, va) and (kb, vb); *sorted_* name the buffers
// holding the result.  K is uint32_t or unsigned long long.
template <typename K>
size_t radix_sort_scratch(int n);
template <typename K>
rtsdf_status radix_sort_pairs(K* ka, uint32_t* va, K* kb, uint32_t* vb, int n, int key_bits, void* scratch,
                              cudaStream_t s, K** sorted_k, uint32_t** sorted_v);

size_t bvh_bytes(int32_t T);
size_t bvh_workspace(int32_t T);
rtsdf_status build_bvh(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid& g,
                       void* bvh, void* ws, rtsdf_counters* counters, cudaStream_t s);

rtsdf_status jfa(const rtsdf_grid& g, int32_t* a, int32_t* b, const int32_t* steps, int32_t nsteps,
                 int32_t** result, cudaStream_t s);

size_t refine_workspace(const rtsdf_grid& g);
rtsdf_status refine(const rtsdf_grid& g, int32_t T, const void* bvh, const int32_t* nearest, const int32_t* rep_tri, const rtsdf_refine_params& p,
                    uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf, void* ws,
                    rtsdf_counters* counters, uint32_t* win_ray, int32_t* win_tri, const rtsdf_grid* coarse,
                    int ratio, cudaStream_t s);

rtsdf_status shadow(const rtsdf_grid& g, const float* sdf, const float* pos, const float* nrm, int32_t P,
                    const rtsdf_shadow_params& p, float* vis, cudaStream_t s);
rtsdf_status shadow_coherent(const rtsdf_grid& g, const float* sdf, const float* pos, const float* nrm, int32_t P,
                             const rtsdf_shadow_params& p, float* vis, uint8_t* steps, cudaStream_t s);

rtsdf_status sample(const rtsdf_grid& g, const float* sdf, const float* pts, int32_t M, float* out, cudaStream_t s);

size_t backward_workspace(const rtsdf_grid& g);
rtsdf_status backward(const rtsdf_grid& g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                      const int32_t* nearest, const int32_t* rep_tri, const uint32_t* front, const uint32_t* back,
                      const uint32_t* win_ray, const int32_t* win_tri, const rtsdf_refine_params& rp,
                      const float* sdf, const float* pts, int32_t M, const float* d_samples, const float* pos,
                      const float* nrm, int32_t P, const rtsdf_shadow_params& sp, const float* d_vis,
                      float* d_verts, float* d_light, void* ws, cudaStream_t s);

}  // namespace rtsdf
