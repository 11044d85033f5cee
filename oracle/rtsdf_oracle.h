/*
 * CPU oracle of the RTSDF hot path (Tan, Chua, Koh, Bhojan, "RTSDF: Real-time
 * Signed Distance Fields for Soft Shadow Approximation in Games").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-pass restatements of each step
 * of the method, used by the tests, the smoke check and the CPU-baseline leg of
 * the benchmark to judge the CUDA library.  Nothing on the product path may call
 * this code, and it shares no code, header or constant table with the CUDA path.
 *
 * Precision: the paper states none.  Every decision that turns floating point
 * into an integer (triangle/box overlap, ray/triangle hit, closest hit, the
 * representative-triangle argmin, raymarch stop) is taken in IEEE FP32, with the
 * operation order written out in the code and no contraction to FMA (build with
 * -ffp-contract=off), because the GPU takes the same decisions in FP32.  FP64
 * restatements that serve as ground truth live in the tests.
 *
 * All geometry is in voxel units: a world point v maps to (v - origin) / h, so the
 * centre of voxel (i, j, k) is exactly (i + 0.5, j + 0.5, k + 0.5).
 */
#ifndef RTSDF_ORACLE_H
#define RTSDF_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t nx, ny, nz;
    float ox, oy, oz;
    float h;
} or_grid;

/* Packed seed of voxel (i, j, k) = (k << 20) | (j << 10) | i; no seed = -1. */
#define OR_EMPTY (-1)

/* world -> voxel coordinates, (v - o) / h per component. */
void or_to_voxel(const float* verts, int32_t V, const or_grid* g, float* out);

/* Closed triangle / closed axis-aligned cube overlap by the separating-axis theorem
 * (13 axes).  Returns 1 on overlap.  Box given by centre and half-size. */
int or_tri_box_overlap(const float* a, const float* b, const float* c,
                       float cx, float cy, float cz, float hs);

/* Squared distance from p to the closest point of triangle abc (Voronoi-region
 * walk, computed in the frame of p). */
float or_closest_d2(const float* p, const float* a, const float* b, const float* c);

/* Sec. 2.2: voxelize at the SDF resolution; seed[v] = packed(v) where a triangle
 * overlaps voxel v, else -1; rep_tri[v] = the overlapping triangle closest to the
 * voxel centre (ties to the lower id), else -1.  vv = voxel-space vertices.
 * Returns the number of skipped (invalid) triangles. */
int32_t or_voxelize(const float* vv, int32_t V, const int32_t* tris, int32_t T,
                    const or_grid* g, int32_t* seed, int32_t* rep_tri);

/* Sec. 2.2: one jump-flooding pass with offset k: every voxel takes, among the 27
 * voxels v + k*d (d in {-1,0,1}^3, inside the grid), the stored seed closest to it
 * (integer squared distance; ties to the lower packed seed). */
void or_jfa_pass(const or_grid* g, const int32_t* in, int32_t k, int32_t* out);

/* Coarse distance (Sec. 2.2 / 2.3): distance from each voxel centre to the
 * representative triangle of its flooded seed; mask (Sec. 2.3): squared integer
 * seed distance <= mask_vox^2.  No seed: u_c = empty_dist, unmasked. */
void or_resolve(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                const int32_t* rep_tri, float mask_vox, float empty_dist,
                float* u_c, uint8_t* mask);

/* Two resolutions (Sec. 2.5.1): resolve fine voxels against the flooded seeds and
 * representative triangles of the coarse grid gc (ratio = fine voxels per coarse
 * voxel); the mask is on the integer seed distance in coarse voxels. */
void or_resolve_2res(const or_grid* gf, const or_grid* gc, int32_t ratio, const float* vv, const int32_t* tris,
                     const int32_t* nearest_c, const int32_t* rep_c, float mask_vox, float empty_dist, float* u_c,
                     uint8_t* mask);
void or_fine_rep_2res(const or_grid* gf, const or_grid* gc, int32_t ratio, const int32_t* nearest_c,
                      const int32_t* rep_c, int32_t* rep_f);

/* Philox4x32-10 (Salmon et al., SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Sec. 2.1: uniform direction on the unit sphere for one ray, Marsaglia (1972)
 * rejection from Philox words.  Returns the attempt that succeeded, or -1. */
int or_sphere_dir(uint32_t voxel, uint32_t ray, uint32_t scene, const uint32_t key[2], float dir[3]);

/* Ray / triangle (Moller-Trumbore).  Hit iff 0 < t <= tmax.  *front = 1 when the
 * ray meets the outward (counter-clockwise) side.  On a hit, *margin (may be NULL)
 * is the smallest of the barycentric coordinates u, w and 1 - (u + w). */
int or_ray_tri(const float o[3], const float d[3], const float* a, const float* b, const float* c,
               float tmax, float* t, int* front, float* margin);

/* Sec. 2.1: ray-sampled refinement of the listed voxels by brute force over all
 * triangles.  For voxel vox[i], rays r = 0..R-1 get ray id frame*R + r; each ray's
 * closest hit (ties to the lower triangle id) lowers dist and votes front/back.
 * dist/front/back hold the incoming state (float bits) and are updated in place.
 * When this call's closest hit (t, then triangle id, then first ray) lowers dist,
 * win_ray/win_tri (may be NULL) record that ray id and triangle: the frozen source
 * of the refined distance used by the adjoint.  *near_edge (may be NULL) gets
 * the number of (ray, triangle) hits, over every triangle, whose barycentric margin
 * is below 1e-6.
 * Returns the number of rays whose direction could not be drawn. */
int64_t or_refine_voxels(const or_grid* g, const float* vv, int32_t V, const int32_t* tris, int32_t T,
                         const int32_t* vox, int64_t n, int32_t R, float tmax,
                         const uint32_t key[2], uint32_t frame, uint32_t scene,
                         uint32_t* dist_bits, uint32_t* front, uint32_t* back,
                         uint32_t* win_ray, int32_t* win_tri, int64_t* near_edge);

/* Sign of a refined voxel (Sec. 2.1): negative iff back > front; on a tie the side
 * of the representative triangle's plane decides when fallback != 0. Returns -1/+1. */
int or_vote_sign(uint32_t front, uint32_t back, const float* p, const float* a, const float* b,
                 const float* c, int fallback);

/* Signed SDF (Sec. 2.1-2.3): masked voxels take the vote sign times the refined
 * distance; the others take the coarse distance minus beta (the thickened,
 * hollow jump-flooded field). */
void or_finalize(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                 const int32_t* rep_tri, const uint8_t* mask, const float* u_c,
                 const uint32_t* dist_bits, const uint32_t* front, const uint32_t* back,
                 float beta, int fallback, float* sdf);

/* Trilinear sample of a voxel-centred grid at voxel coordinate q (clamp to edge). */
float or_trilinear(const or_grid* g, const float* sdf, float qx, float qy, float qz);

/* The field at M world points: q = (p - o) / h per component, then trilinear. */
void or_sample(const or_grid* g, const float* sdf, const float* pts, int32_t M, float* out);

/* Sec. 2.4 / 2.5.2: soft-shadow visibility of P receivers (world positions and
 * unit normals) toward a directional light, sphere tracing the SDF (voxel units). */
void or_shadow(const or_grid* g, const float* sdf, const float* pos, const float* nrm, int32_t P,
               const float light_dir[3], float k, int32_t steps, float max_step, float start_off,
               float normal_off, float hit_eps, float bias, const float* t_start, float* vis);

/* Sec. 2.5.2 jitter: per-receiver first-sample distances start_off + jitter * u_i
 * (u_i from Philox4x32-10 on counter (i, frame, 0x4A177E2, 0), key (0x51AD0, 0x7E2)).
 * or_shadow and or_shadow_loss_f64 take them in t_start (NULL: start_off). */
void or_jitter_starts(int32_t P, float start_off, float jitter, uint32_t frame, float* t_start);

/* ------------------------------------------------------------------ adjoint (FP64) */

/* Frozen source of a voxel's field value (rtsdf_oracle_adjoint.c). */
enum { OR_SRC_CONST = 0, OR_SRC_COARSE_UNMASKED = 1, OR_SRC_COARSE_MASKED = 2, OR_SRC_RAY = 3 };
typedef struct {
    int32_t kind;  /* OR_SRC_* */
    int32_t tri;   /* representative triangle (coarse) or hit triangle (ray) */
    float sign;    /* vote sign of a masked voxel */
    float dir[3];  /* direction of the winning ray */
} or_src;

/* Freezes every discrete choice of a forward pass: flooded seed's representative
 * triangle, mask, vote sign and the source of a refined distance (win_ray ==
 * 0xFFFFFFFF: the coarse closest point; else that ray's hit of win_tri). */
void or_frozen_sources(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                       const int32_t* rep_tri, const uint8_t* mask, const uint32_t* front, const uint32_t* back,
                       const uint32_t* win_ray, const int32_t* win_tri, const uint32_t key[2], uint32_t scene,
                       int fallback, or_src* out);

/* The frozen field in FP64 for world-space vertices (voxel units) and the
 * accumulation of dL/d(world vertex) from dL/d(field). */
void or_frozen_sdf_f64(const or_grid* g, const double* verts, const int32_t* tris, const or_src* src, double beta,
                       double* sdf);
void or_frozen_sdf_backward_f64(const or_grid* g, const double* verts, const int32_t* tris, const or_src* src,
                                double beta, const double* gsdf, double* gverts);

/* sum_m (trilinear(field, pts_m) - target_m)^2 in FP64; adds dL/d(field) when gsdf != NULL. */
double or_sample_loss_f64(const or_grid* g, const double* sdf, const float* pts, int32_t M, const float* target,
                          double* gsdf);

/* sum_p (vis_p - target_p)^2 of the soft-shadow raymarch with the control flow of
 * the FP32 march on sdf32 toward l_decide and the values of the FP64 field sdf
 * toward l; adds dL/d(field) and dL/d(light direction l, unnormalised) when the
 * pointers are not NULL. */
double or_shadow_loss_f64(const or_grid* g, const float* sdf32, const double* sdf, const float* pos,
                          const float* nrm, int32_t P, const float l_decide[3], const double l[3], float k,
                          int32_t steps, float max_step, float start_off, float normal_off, float hit_eps,
                          float bias, const float* t_start, const float* target, double* gsdf, double* gl);

/* Helpers for the tests: number of OpenMP threads the oracle uses. */
/* OpenMP threads of the voxel-parallel loops (the timing baseline sets 1 or all). */
void or_set_num_threads(int n);
int or_num_threads(void);

#endif
