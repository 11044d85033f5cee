/*
 * rtsdf.h -- C-ABI of librtsdf, a GB300 (sm_103a) implementation of the per-frame
 * signed-distance-field rebuild and soft-shadow raymarch of RTSDF (Tan, Chua,
 * Koh, Bhojan: "RTSDF: Real-time Signed Distance Fields for Soft Shadow
 * Approximation in Games").
 *
 * Pipeline per frame (Sec. 2): conservative voxelization of the triangle scene
 * into a seed grid (rtsdf_voxelize) -> 3D jump flooding of nearest seeds
 * (rtsdf_jfa) -> ray-sampled refinement of voxels close to a surface, with
 * a device-built BVH (rtsdf_build_bvh, rtsdf_refine) -> sphere-traced soft shadow
 * on the resulting field (rtsdf_shadow).
 *
 * Conventions shared by every call
 *  - Grid: nx*ny*nz voxels (each dimension 1..1023) of edge h, min corner origin;
 *    linear index (k*ny + j)*nx + i, x fastest.  World point v maps to voxel
 *    coordinates (v - origin)/h, so voxel (i,j,k) has its centre at (i+.5,j+.5,k+.5).
 *    Distances in parameters and outputs are in voxel units.
 *  - Packed seed: (k << 20) | (j << 10) | i; RTSDF_EMPTY (-1) = no seed.
 *  - Meshes: float32 vertices [V][3] (world), int32 triangles [T][3], counter-
 *    clockwise seen from outside.  Triangles with an index outside [0, V) or a
 *    non-finite vertex are skipped by every call (and counted).
 *  - Memory: every pointer argument is DEVICE memory owned by the caller unless
 *    stated otherwise; the library never allocates, frees or synchronises.  Work
 *    is enqueued on `stream` (NULL = legacy default stream).  Workspaces are
 *    caller-allocated, sized by the matching *_workspace query, 256-byte aligned.
 *  - Errors: return codes only.  Argument errors are reported before anything is
 *    enqueued (RTSDF_EINVAL / RTSDF_ENOMEM); launch failures as RTSDF_ECUDA.
 *    Device-side conditions (skipped triangles, traversal-stack overflow, rays
 *    whose direction could not be drawn) are counted in an optional rtsdf_counters
 *    block in device memory that the caller zeroes and reads back.
 *  - Determinism: every output is independent of scheduling; integer outputs are
 *    bit-exact against the plain definitions (no FMA contraction, correctly
 *    rounded division and square root).
 */
#ifndef RTSDF_H
#define RTSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* rtsdf_stream;

#define RTSDF_EMPTY (-1)
#define RTSDF_MAX_DIM 1023

typedef enum {
    RTSDF_OK = 0,
    RTSDF_EINVAL = 1, /* invalid argument (null or misaligned pointer, bad size or parameter) */
    RTSDF_ENOMEM = 2, /* caller-provided workspace or buffer smaller than required */
    RTSDF_ECUDA = 3   /* a CUDA launch or runtime call failed */
} rtsdf_status;

typedef struct {
    int32_t nx, ny, nz; /* voxels per axis, 1..1023 */
    float origin[3];    /* world position of the grid's min corner */
    float h;            /* voxel edge in world units, > 0 */
} rtsdf_grid;

/* Ray-sampled refinement (Sec. 2.1) and ray mask (Sec. 2.3); distances in voxels. */
typedef struct {
    float mask_vox;         /* refine voxel v iff |v - seed(v)|^2 <= mask_vox^2 (integer seed distance) */
    int32_t rays_per_voxel; /* R >= 1 rays per masked voxel per call */
    float max_ray_vox;      /* a hit counts iff 0 < t <= max_ray_vox */
    float beta_vox;         /* unmasked voxels store coarse distance - beta (Sec. 2.2 thickening) */
    uint32_t key[2];        /* Philox4x32-10 key */
    uint32_t frame_index;   /* ray r of this call has ray id frame_index*R + r */
    uint32_t scene_id;      /* third Philox counter word */
    int32_t accumulate;     /* 0: fresh; 1: keep the minimum and the votes of earlier frames (Sec. 2.1
                               temporal accumulation); 2: decayed accumulation of Eq. (1), see rtsdf_refine */
    int32_t sign_fallback;  /* 1: front == back -> side of the representative triangle's plane */
    float decay_alpha;      /* alpha of Eq. (1) (accumulate = 2), in [0, 1] */
    int32_t count_work;     /* nonzero: also count the work units and near-edge hits of the ray sampling
                               into the counters' node_tests ... exact_tests and near_edge_hits (about 3%
                               slower; rtsdf_refine_tracked and the batch never count them) */
} rtsdf_refine_params;

/* Soft-shadow raymarch (Sec. 2.4, 2.5.2, 2.5.3); distances in voxels. */
typedef struct {
    float light_dir[3];      /* direction toward the light (normalised by the library) */
    float k;                 /* penumbra factor */
    int32_t steps;           /* maximum samples per receiver */
    float max_step_vox;      /* step cap (Sec. 2.5.2) */
    float start_offset_vox;  /* first sample distance along the light direction */
    float normal_offset_vox; /* lift of the ray origin along the receiver normal */
    float hit_eps_vox;       /* occluded when sampled distance <= hit_eps */
    float bias_vox;          /* subtracted from every sample (Sec. 2.5.3 thickening) */
    float jitter_vox;        /* Sec. 2.5.2 jitter: receiver i starts at start_offset + jitter * u_i */
    uint32_t frame_index;    /* u_i in [0, 1) from Philox4x32-10 on counter (i, frame_index, 0x4A177E2, 0),
                                key (0x51AD0, 0x7E2): the top 24 bits of the first word times 2^-24 */
    const float* light_dir_device; /* NULL, or a DEVICE pointer (4-byte aligned) to 3 floats used instead
                                      of light_dir: read by the kernels when they run (stream order), so
                                      a light that lives on the GPU (a trained parameter) needs no copy to
                                      the host; normalised on the device with the same FP32 operations.
                                      Not validated: a zero or non-finite vector gives NaN visibilities. */
} rtsdf_shadow_params;

/* Device-side counters; each call adds to the fields it owns.  The caller zeroes
 * the block and reads it back; it must be 8-byte aligned.  The 64-bit fields count
 * the refinement's work (Sec. 2.1), for throughput figures:
 *   node_tests   BVH child boxes tested against a brick's reach region (or, for the
 *                bricks of a coarse grid that walk each ray on its own, against a ray),
 *   reach_tests  (masked voxel, staged triangle) pairs tested for reach,
 *   filter_pairs pairs within reach, each then filtered against every ray of the voxel,
 *   exact_tests  (ray, triangle) pairs given the exact Moller-Trumbore test.
 * near_edge_hits counts the exact-test hits whose smallest barycentric coordinate
 * (u, w or 1 - u - w, as the test computes them in FP32) is below 1e-6: the hits a
 * different rounding of the same arithmetic could turn into misses.  It counts hits
 * over every tested triangle, not only each ray's closest, so it equals the count
 * of a brute-force test of every (ray, triangle) pair. */
typedef struct {
    uint32_t skipped_triangles; /* voxelize / build_bvh: invalid triangles */
    uint32_t masked_voxels;     /* refine: voxels inside the ray mask */
    uint32_t rays_hit;          /* refine: rays with a hit */
    uint32_t rays_failed;       /* refine: rays with no direction after 32 Philox draws */
    uint32_t stack_overflow;    /* refine: traversals that overflowed the stack (result incomplete) */
    uint32_t near_edge_hits;    /* refine: exact-test hits within 1e-6 (barycentric) of an edge */
    uint32_t reserved[2];
    uint64_t node_tests;        /* refine: BVH child-box tests */
    uint64_t reach_tests;       /* refine: (voxel, triangle) reach tests */
    uint64_t filter_pairs;      /* refine: (voxel, triangle) pairs filtered against the voxel's rays */
    uint64_t exact_tests;       /* refine: exact ray/triangle tests */
} rtsdf_counters;

/* ---------------------------------------------------------------- voxelize */

/* Bytes of workspace rtsdf_voxelize needs for T triangles on grid g (0 on bad args). */
size_t rtsdf_voxelize_workspace(int32_t T, const rtsdf_grid* g);

/* Sec. 2.2 (Jump Flooding): "we voxelize the scene with voxel resolution equal to
 * our final distance field", every triangle point being a seed.  Conservative:
 * voxel v is a seed iff some closed triangle overlaps v's closed cube (13-axis
 * separating-axis test in FP32).  Outputs (nx*ny*nz int32 each):
 *   seed[v]    = packed(v) for seed voxels, else RTSDF_EMPTY;
 *   rep_tri[v] = among the triangles overlapping v, the one whose closest point is
 *                nearest v's centre (ties -> lower triangle id); -1 elsewhere.
 * ws >= rtsdf_voxelize_workspace(T, g).  counters may be NULL. */
rtsdf_status rtsdf_voxelize(const float* verts, int32_t V, const int32_t* tris, int32_t T,
                            const rtsdf_grid* g, int32_t* seed, int32_t* rep_tri,
                            void* ws, size_t ws_bytes, rtsdf_counters* counters, rtsdf_stream stream);

/* ---------------------------------------------------------------- BVH */

/* Bytes of the BVH buffer and of the build workspace for T triangles. */
size_t rtsdf_bvh_bytes(int32_t T);
size_t rtsdf_bvh_workspace(int32_t T);

/* Bounding-volume hierarchy over the mesh for the ray queries of Sec. 2.1 (the
 * paper uses the driver-built DXR structure, Sec. 2 and 3.5.1): linear BVH from
 * 30-bit Morton codes of triangle centroids in the grid box, radix-sorted, with
 * Karras' (HPG 2012) radix-tree topology and bottom-up conservative boxes.  The
 * buffer is self-contained (leaves hold voxel-space triangles for the ray tests,
 * and a table indexed by triangle id holds each triangle's voxel-space vertices,
 * which rtsdf_refine's coarse distance and sign fallback read) and only
 * meaningful to rtsdf_refine with the same mesh and grid. */
rtsdf_status rtsdf_build_bvh(const float* verts, int32_t V, const int32_t* tris, int32_t T,
                             const rtsdf_grid* g, void* bvh, size_t bvh_bytes,
                             void* ws, size_t ws_bytes, rtsdf_counters* counters, rtsdf_stream stream);

/* ---------------------------------------------------------------- BVH, no allocation */

/* Largest mesh rtsdf_build_bvh_noalloc accepts, and the device memory its fixed
 * scratch array occupies on every GPU that loads this library, until exit. */
#define RTSDF_NOALLOC_MAX_TRIS 131072
#define RTSDF_NOALLOC_SCRATCH_BYTES (4u << 20)

/* No counterpart in the paper: a convenience of this library.  rtsdf_build_bvh
 * without a caller workspace, for hosts that cannot allocate device memory on the
 * library's behalf, e.g. an engine whose memory manager owns the GPU and forbids
 * cudaMalloc inside its frame loop (cudaMalloc can synchronise the device and stall
 * the frame).  Its scratch is one fixed array in device memory inside the library;
 * the call itself allocates nothing.  The caller still passes the mesh and the
 * output BVH buffer; arguments, outputs and errors are those of rtsdf_build_bvh, and
 * T > RTSDF_NOALLOC_MAX_TRIS returns RTSDF_ENOMEM.
 * The first call on a device looks up the array's device address (one-time set-up
 * per device, with that device current; looked up again if the device's context
 * has changed since, e.g. after cudaDeviceReset); make that first call before any
 * stream capture.  Every call on a device uses the same array, which keeps the previous
 * call's contents (the build clears what must start at zero): calls that can
 * overlap on the GPU (other streams, other host threads) race, so the caller must
 * serialise them. */
rtsdf_status rtsdf_build_bvh_noalloc(const float* verts, int32_t V, const int32_t* tris, int32_t T,
                                     const rtsdf_grid* g, void* bvh, size_t bvh_bytes,
                                     rtsdf_counters* counters, rtsdf_stream stream);

/* ---------------------------------------------------------------- jump flooding */

/* Sec. 2.2 (Jump Flooding, after Rong & Tan 2006, extended to 3D): for each
 * offset k = steps[0], steps[1], ... every voxel v takes, among the stored seeds
 * of the 27 voxels v + k*d, d in {-1,0,1}^3 inside the grid, the one nearest v
 * (integer squared distance between voxel centres; ties -> lower packed seed).
 * Passes read one buffer and write the other (Jacobi).  buf_a holds the seeds on
 * entry; both buffers are nx*ny*nz int32.  On return *result (host pointer) names
 * the buffer that holds the flooded field (buf_a for an even number of passes).
 * steps: HOST array of nsteps offsets, each in 1..1023; nsteps >= 0. */
rtsdf_status rtsdf_jfa(const rtsdf_grid* g, int32_t* buf_a, int32_t* buf_b, const int32_t* steps,
                       int32_t nsteps, int32_t** result, rtsdf_stream stream);

/* ---------------------------------------------------------------- refine */

size_t rtsdf_refine_workspace(const rtsdf_grid* g);

/* Coarse field, ray mask and ray-sampled refinement of one frame.
 *  - Coarse (Sec. 2.2-2.3): u_c(v) = distance from v's centre to rep_tri of its
 *    flooded seed nearest(v); mask(v) iff integer |v - nearest(v)|^2 <= mask_vox^2.
 *    Unmasked voxels get sdf_out = u_c - beta (no seed: u_c = nx+ny+nz).
 *  - Refine (Sec. 2.1): each masked voxel shoots R rays from its centre with
 *    directions uniform on the sphere (Philox4x32-10 on counter (voxel, ray id,
 *    scene_id, attempt) + Marsaglia's rejection method).  The closest hit of each
 *    ray (0 < t <= max_ray_vox, ties -> lower triangle id) lowers dist and adds a
 *    front (ray meets the counter-clockwise side) or back vote.
 *  - State: dist_bits (float bits), front, back are nx*ny*nz uint32.  Unmasked
 *    voxels get (u_c, 0, 0).  At masked voxels accumulate = 0 starts them at
 *    (u_c, 0, 0); accumulate = 1 keeps earlier frames (dist = min(dist, u_c), votes
 *    kept); accumulate = 2 is Eq. (1) (Sec. 2.5.1): dist = alpha * f + (1 - alpha) *
 *    u_c with f the previous frame's dist, then the minimum with this frame's hits;
 *    votes are this frame's only.
 *  - sdf_out (nx*ny*nz float) at masked voxels: -dist if back > front, +dist if
 *    front > back; on a tie the side of rep_tri's plane when sign_fallback, else +.
 * verts/tris must be the mesh the BVH and rep_tri were built from. */
rtsdf_status rtsdf_refine(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris,
                          int32_t T, const void* bvh, size_t bvh_bytes, const int32_t* nearest,
                          const int32_t* rep_tri, const rtsdf_refine_params* p, uint32_t* dist_bits,
                          uint32_t* front, uint32_t* back, float* sdf_out, void* ws, size_t ws_bytes,
                          rtsdf_counters* counters, rtsdf_stream stream);

/* Refinement that also records, per voxel, the source that set its distance (the
 * winner), for rtsdf_backward.  Arguments, outputs and errors are those of
 * rtsdf_refine, plus two nx*ny*nz arrays (device, 16-byte aligned, both non-NULL):
 *   win_ray[v] = ray id (frame_index*R + r) of the hit that set dist[v], or
 *                0xFFFFFFFF when the coarse distance u_c holds it (always at
 *                unmasked voxels);
 *   win_tri[v] = that hit's triangle id, or -1.
 * Among this call's rays the winner is the smallest (t, triangle id), the first
 * ray on ties; it replaces the record only when it lowers dist.  With accumulate
 * = 0 every record starts at the coarse source; with accumulate = 1 the coarse
 * source takes over a voxel when u_c lowers its distance. */
rtsdf_status rtsdf_refine_tracked(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris,
                                  int32_t T, const void* bvh, size_t bvh_bytes, const int32_t* nearest,
                                  const int32_t* rep_tri, const rtsdf_refine_params* p, uint32_t* dist_bits,
                                  uint32_t* front, uint32_t* back, float* sdf_out, uint32_t* win_ray,
                                  int32_t* win_tri, void* ws, size_t ws_bytes, rtsdf_counters* counters,
                                  rtsdf_stream stream);

/* Two resolutions (Sec. 2.5.1: JFA on a coarse grid, e.g. 128^3, the refined field on
 * a fine grid, e.g. 256^3).  Same as rtsdf_refine on the FINE grid `fine` (state,
 * sdf_out and workspace are fine grids; the BVH is built for the fine grid), except
 * that `nearest` (flooded seeds) and `rep_tri` are grids of `coarse`: fine voxel
 * (i,j,k) takes the seed of coarse voxel (i/r, j/r, k/r), r = coarse h / fine h (a
 * positive integer, same origin, coarse dims = ceil(fine dims / r), else
 * RTSDF_EINVAL); u_c is the distance from the fine voxel's centre to that seed's
 * representative triangle; the mask compares the integer seed distance in COARSE
 * voxels with mask_vox^2 (mask_vox in coarse voxels).  beta_vox and max_ray_vox are
 * in fine voxels.  rtsdf_backward supports single-resolution fields only. */
rtsdf_status rtsdf_refine_2res(const rtsdf_grid* fine, const rtsdf_grid* coarse, const float* verts, int32_t V,
                               const int32_t* tris, int32_t T, const void* bvh, size_t bvh_bytes,
                               const int32_t* nearest, const int32_t* rep_tri, const rtsdf_refine_params* p,
                               uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf_out, void* ws,
                               size_t ws_bytes, rtsdf_counters* counters, rtsdf_stream stream);

/* ---------------------------------------------------------------- shadow */

/* Sec. 2.4 sphere tracing toward a directional light with the penumbra estimate
 * k * e / (t - y) (Sec. 2.4; Aaltonen 2018 triangulation of the two latest samples,
 * Sec. 2.5.2: y = d^2 / (2 d_prev), e = sqrt(d^2 - y^2)), step cap (Sec. 2.5.2),
 * bias (Sec. 2.5.3).  The SDF is sampled trilinearly between voxel centres (clamp
 * to edge).  Receiver i: world position pos[3i..], normal nrm[3i..] (the headless
 * stand-in for a G-buffer).  Marching stops when the sample leaves the grid box,
 * after `steps` samples, or when the sample is <= hit_eps (visibility 0).
 * vis[i] in [0, 1]. */
rtsdf_status rtsdf_shadow(const rtsdf_grid* g, const float* sdf, const float* pos, const float* nrm,
                          int32_t P, const rtsdf_shadow_params* p, float* vis, rtsdf_stream stream);

/* rtsdf_shadow with the receivers regrouped for SIMT coherence (the same vis bit for
 * bit: each receiver's march is independent of the others).  steps (P bytes of device
 * memory, caller-owned, kept from call to call for the same receivers; zeroes the
 * first time) holds each receiver's march length from the previous call: the step at
 * which its march stopped, at most 255.  Within each block of 512 consecutive
 * receivers the threads take the receivers in order of those lengths, so the lanes
 * of a warp march about as long; every receiver's new length is written back.  Any
 * contents of steps give the same vis; only the speed depends on them.  EINVAL as
 * rtsdf_shadow, or when steps is NULL with P > 0. */
rtsdf_status rtsdf_shadow_coherent(const rtsdf_grid* g, const float* sdf, const float* pos, const float* nrm,
                                   int32_t P, const rtsdf_shadow_params* p, float* vis, uint8_t* steps,
                                   rtsdf_stream stream);

/* ---------------------------------------------------------------- shadow, texture path */

/* The shadow raymarch sampling the field through a 3D texture with hardware
 * trilinear filtering (Sec. 2.1 notes the 3D-texture grid allows hardware
 * interpolation).  rtsdf_texture_create allocates the texture's CUDA array (nx*ny*nz
 * floats) on the current device -- this object, like a batch plan, is owned by the
 * library and freed by rtsdf_texture_destroy; rtsdf_texture_upload copies a field
 * (device, x fastest) into it on `stream`.  rtsdf_shadow_tex is rtsdf_shadow with the
 * texture's field; the texture unit's weights have 8 fractional bits, so samples
 * differ from the FP32 lerps by up to about 1/256 of the difference between
 * neighbouring voxels and visibilities differ from rtsdf_shadow's (measured: mean
 * absolute difference about 4e-5, 99.9% of receivers within 1.3e-3; a receiver whose
 * hit decision flips can differ by more). */
typedef struct rtsdf_texture rtsdf_texture;
rtsdf_status rtsdf_texture_create(const rtsdf_grid* g, rtsdf_texture** tex);
void rtsdf_texture_destroy(rtsdf_texture* tex);
rtsdf_status rtsdf_texture_upload(rtsdf_texture* tex, const float* sdf, rtsdf_stream stream);
rtsdf_status rtsdf_shadow_tex(const rtsdf_texture* tex, const float* pos, const float* nrm, int32_t P,
                              const rtsdf_shadow_params* p, float* vis, rtsdf_stream stream);

/* ---------------------------------------------------------------- field samples */

/* The field at M world points pts[3m..] (voxel coordinates (p - origin)/h, then
 * trilinear between voxel centres with clamp to edge, FP32 lerps in x, y, z: the
 * sampling the shadow raymarch of Sec. 2.4 uses).  out: M floats (voxel units). */
rtsdf_status rtsdf_sample(const rtsdf_grid* g, const float* sdf, const float* pts, int32_t M, float* out,
                          rtsdf_stream stream);

/* ---------------------------------------------------------------- adjoint */

/* Longest raymarch (rtsdf_shadow_params.steps) rtsdf_backward replays. */
#define RTSDF_BACKWARD_MAX_STEPS 512

size_t rtsdf_backward_workspace(const rtsdf_grid* g);

/* No counterpart in the paper: the adjoint of the forward outputs
 *   samples = rtsdf_sample(sdf, pts)            (M values)
 *   vis     = rtsdf_shadow(sdf, pos, nrm, sp)   (P values)
 * with respect to the mesh vertices (world units) and the light direction
 * sp->light_dir (unnormalised, as passed), given upstream gradients d_samples (M)
 * and d_vis (P).  The field is the one the forward built on this grid from
 * verts/tris: nearest (flooded seeds), rep_tri (voxelizer), front/back (votes) and
 * win_ray/win_tri (rtsdf_refine_tracked) after its last frame, with the refine
 * parameters rp of that frame (mask, key, scene_id, sign_fallback; the voxel's ray
 * id in win_ray already includes the frame).  Every discrete choice of the forward
 * is held fixed: the representative triangle, the mask, the vote, the winning
 * source, and the raymarch's control flow; the adjoint is the exact derivative of
 * that frozen function:
 *   coarse voxels (Sec. 2.2): d|q - p| / dX_m = lambda_m (q - p)/|q - p| (closest
 *     point q with barycentric weights lambda);
 *   refined voxels (Sec. 2.1): dt / dX_m = lambda_m n / (d . n) (hit t of the
 *     winning ray d on its triangle, normal n, weights lambda of the hit point);
 *   samples: trilinear weights; shadow (Sec. 2.4, 2.5.2): reverse mode through the
 *     replayed march and the penumbra estimate at its minimising sample.
 * Outputs (overwritten): d_verts [V][3], d_light [3], both device float.  The FP32
 * sums are accumulated with atomics, so the last bits vary between runs.
 * pts/d_samples may be NULL when M = 0, pos/nrm/d_vis when P = 0.
 * sp->steps > RTSDF_BACKWARD_MAX_STEPS -> RTSDF_EINVAL.
 * ws >= rtsdf_backward_workspace(g). */
rtsdf_status rtsdf_backward(const rtsdf_grid* g, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                            const int32_t* nearest, const int32_t* rep_tri, const uint32_t* front,
                            const uint32_t* back, const uint32_t* win_ray, const int32_t* win_tri,
                            const rtsdf_refine_params* rp, const float* sdf, const float* pts, int32_t M,
                            const float* d_samples, const float* pos, const float* nrm, int32_t P,
                            const rtsdf_shadow_params* sp, const float* d_vis, float* d_verts, float* d_light,
                            void* ws, size_t ws_bytes, rtsdf_stream stream);

/* ---------------------------------------------------------------- batched rebuild */

/* No counterpart in the paper: many scenes of different grid sizes and meshes
 * rebuilt together (voxelize, BVH, jump flooding, coarse field + ray mask,
 * refinement; the steps of rtsdf_voxelize .. rtsdf_refine) with one launch per
 * step for the whole batch instead of one per scene, the JFA pass chain replayed
 * from a captured CUDA graph, and the refinement's brick shape and warps per CTA
 * chosen by rtsdf_batch_autotune.  Every scene's outputs are bit-identical to its
 * own single-scene calls with the same parameters. */

#define RTSDF_BATCH_MAX_SCENES 64
#define RTSDF_BATCH_MAX_STEPS 16

typedef struct {
    rtsdf_grid grid;
    int32_t V, T;                         /* vertices and triangles of this scene's mesh */
    int32_t nsteps;                       /* JFA offsets of this scene, 0..RTSDF_BATCH_MAX_STEPS */
    int32_t steps[RTSDF_BATCH_MAX_STEPS]; /* each 1..1023, as rtsdf_jfa's steps */
    rtsdf_refine_params refine;           /* frame_index and accumulate are set per rebuild call */
} rtsdf_batch_scene;

/* Where a scene lives in the batch's buffers (computed by the plan). */
typedef struct {
    int64_t voxel_offset;    /* first voxel in every batch grid array (a multiple of 64) */
    int32_t vertex_offset;   /* first vertex in the batch vertex array */
    int32_t triangle_offset; /* first triangle in the batch triangle array; its indices are local to the scene */
    int64_t bvh_offset;      /* byte offset of the scene's BVH in the batch BVH buffer (256-aligned) */
    int32_t flooded_in_b;    /* 1: the scene's flooded seeds end in buf_b, 0: in seed/buf_a */
    int32_t reserved;
} rtsdf_batch_layout;

/* Refinement launch shape: bricks of brick_x * brick_y * brick_z = 64 voxels
 * (brick_x in {4,8,16,32}, brick_y and brick_z in {1,2,4}), warps_per_cta in
 * {1,2,4}; use_graph = 1 replays the JFA chain from a captured CUDA graph. */
typedef struct {
    int32_t brick_x, brick_y, brick_z;
    int32_t warps_per_cta;
    int32_t use_graph;
} rtsdf_batch_tuning;

/* Device buffers of a batch (all caller-owned; grid arrays hold rtsdf_batch_voxels
 * elements, laid out per rtsdf_batch_layout). */
typedef struct {
    const float* verts;  /* [sum V][3] world, scene by scene */
    const int32_t* tris; /* [sum T][3], indices local to each scene's vertices */
    int32_t* seed;       /* in: nothing; out: voxelizer seeds, then JFA ping-pong buffer a */
    int32_t* buf_b;      /* JFA ping-pong buffer b */
    int32_t* rep_tri;    /* representative triangles (ids local to the scene) */
    void* bvh;           /* rtsdf_batch_bvh_bytes bytes */
    size_t bvh_bytes;
    uint32_t* dist_bits; /* refinement state, as rtsdf_refine */
    uint32_t* front;
    uint32_t* back;
    float* sdf;          /* signed field */
    void* ws;            /* rtsdf_batch_workspace bytes */
    size_t ws_bytes;
} rtsdf_batch_buffers;

typedef struct rtsdf_batch_plan rtsdf_batch_plan;

/* Host-only: validates the scenes (1..RTSDF_BATCH_MAX_SCENES) and lays them out.
 * The plan owns host memory, and after the first rebuild a CUDA stream and graph;
 * destroy it with rtsdf_batch_plan_destroy.  It may be used from one host thread
 * at a time. */
rtsdf_status rtsdf_batch_plan_create(const rtsdf_batch_scene* scenes, int32_t S, rtsdf_batch_plan** plan);
void rtsdf_batch_plan_destroy(rtsdf_batch_plan* plan);

rtsdf_status rtsdf_batch_layout_of(const rtsdf_batch_plan* plan, int32_t scene, rtsdf_batch_layout* out);
size_t rtsdf_batch_voxels(const rtsdf_batch_plan* plan);
size_t rtsdf_batch_bvh_bytes(const rtsdf_batch_plan* plan);
size_t rtsdf_batch_workspace(const rtsdf_batch_plan* plan);
rtsdf_status rtsdf_batch_get_tuning(const rtsdf_batch_plan* plan, rtsdf_batch_tuning* out);
rtsdf_status rtsdf_batch_set_tuning(rtsdf_batch_plan* plan, const rtsdf_batch_tuning* t);

/* One frame of every scene: voxelize, BVH, JFA (each scene's own steps, aligned so
 * that all scenes end on the last pass), coarse field and ray mask, refinement with
 * ray ids frame_index*R + r and the given accumulate mode (0, 1, 2 as in
 * rtsdf_refine_params; mode 2 takes each scene's decay_alpha).  counters may be NULL
 * (batch totals).  If the JFA graph is used, the first call with a given pair of
 * JFA buffers captures it (on a stream of the plan) and later calls replay it. */
rtsdf_status rtsdf_batch_rebuild(rtsdf_batch_plan* plan, const rtsdf_batch_buffers* b, uint32_t frame_index,
                                 int32_t accumulate, rtsdf_counters* counters, rtsdf_stream stream);

/* Times the refinement step of the batch under every supported tuning (reps
 * launches each, after one rebuild with the current tuning), keeps the fastest in
 * the plan and returns its time in *best_ms (host pointer, may be NULL).
 * Synchronises the stream.  Leaves the buffers holding a frame-0 rebuild. */
rtsdf_status rtsdf_batch_autotune(rtsdf_batch_plan* plan, const rtsdf_batch_buffers* b, int32_t reps,
                                  float* best_ms, rtsdf_stream stream);

/* ---------------------------------------------------------------- misc */

const char* rtsdf_status_string(rtsdf_status s);

/* Library version as 10000*major + 100*minor + patch. */
int32_t rtsdf_version(void);

/* Number of CUDA kernels this library has enqueued in this process (all devices,
 * all streams), for accounting of launches per frame.  Thread-safe. */
uint64_t rtsdf_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* RTSDF_H */
