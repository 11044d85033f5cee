// Batched rebuild: the voxelize / BVH / jump-flooding / coarse field / refinement
// steps for up to RTSDF_BATCH_MAX_SCENES scenes of different sizes, one launch per
// step for the whole batch.
//
// Every kernel takes the scene table by value (__grid_constant__, a few KB of
// kernel parameters) and maps its flat work index to a scene with a binary search
// over the table's offsets: triangles for the voxelizer and the BVH, voxels for the
// finalisation, thread blocks for the jump flooding and the coarse field, and the
// brick list entries (scene << 25 | brick) for the refinement.  Each scene's
// computation is exactly its single-scene one (the same device functions on the
// scene's slices), so every output is bit-identical to the single-scene calls.
//
// The JFA pass chain (the passes of all scenes aligned so that they end together)
// is captured once into a CUDA graph per pair of ping-pong buffers and replayed.
// The refinement is instantiated for several brick shapes and launched with 1, 2
// or 4 warps per CTA; rtsdf_batch_autotune times them and keeps the fastest.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "bvh_core.cuh"
#include "jfa_core.cuh"
#include "refine_core.cuh"
#include "rtsdf_launch.cuh"
#include "voxelize_core.cuh"

namespace rtsdf {

constexpr int kMaxBatch = RTSDF_BATCH_MAX_SCENES;
constexpr int kBrickBits = 25;  // brick index bits of a work-list entry
constexpr int kVoxChunk = 32;   // (triangle, brick) items per warp chunk (one per lane)

struct SceneD {
    GridD g;
    int32_t V, T, vert_off, tri_off;
    int64_t vox_off, bvh_off, brick_off;
    int32_t tile_start;  // first 32x4x4 resolve tile of the scene in the batch
    int32_t flood_b;     // flooded seeds in buffer b
    float mask2, beta, empty_dist, tmax, alpha;
    int32_t R, fallback;
    uint32_t k0, k1, scene;
    int32_t pad;
};

struct BatchTable {
    int32_t n;
    int32_t nbx_div, nby_div, nbz_div;  // brick shape of this launch (refine only)
    SceneD s[kMaxBatch];
};

// last scene whose start <= x (starts ascending from 0; empty scenes share the
// next scene's start and are skipped)
#define RTSDF_FIND_SCENE(table, field, x)                               \
    ([&]() {                                                            \
        int lo_ = 0, hi_ = (table).n - 1;                               \
        while (lo_ < hi_) {                                             \
            const int mid_ = (lo_ + hi_ + 1) >> 1;                      \
            if ((int64_t)(table).s[mid_].field <= (int64_t)(x)) lo_ = mid_; \
            else hi_ = mid_ - 1;                                        \
        }                                                               \
        return lo_;                                                     \
    }())

// ------------------------------------------------------------------ voxelize

__global__ void k_bvox_count(const __grid_constant__ BatchTable t, const float* __restrict__ verts,
                             const int32_t* __restrict__ tris, int Ttot, uint32_t* __restrict__ counts,
                             rtsdf_counters* counters) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= Ttot) return;
    const SceneD& S = t.s[RTSDF_FIND_SCENE(t, tri_off, gt)];
    float3 a, b, c;
    uint32_t n = 0;
    if (!load_tri(verts + 3 * (int64_t)S.vert_off, S.V, tris + 3 * (int64_t)S.tri_off, gt - S.tri_off, S.g, a, b,
                  c)) {
        if (counters) atomicAdd(&counters->skipped_triangles, 1u);
    } else {
        TriRange r;
        if (tri_range(a, b, c, S.g, r)) n = range_bricks(r);
    }
    counts[gt] = n;
}

__global__ void __launch_bounds__(256, 3) k_bvox_test(const __grid_constant__ BatchTable t,
                                                   const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                                   int Ttot, const uint64_t* __restrict__ offsets,
                                                   unsigned long long* __restrict__ keys) {
    const int64_t warp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / kWarp;
    const uint64_t total = offsets[Ttot];
    const uint64_t nchunks = (total + kVoxChunk - 1) / kVoxChunk;
    for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
        const uint64_t i0 = ch * kVoxChunk, i1 = (i0 + kVoxChunk < total) ? i0 + kVoxChunk : total;
        int lo = 0, hi = Ttot - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i0) lo = mid; else hi = mid - 1;
        }
        vox_chunk<false>(Ttot, offsets, i0, (int)(i1 - i0), lo,
                  [&](int gt, float3& a, float3& b, float3& c, TriRange& r, int& tnx, int& tny,
                      unsigned long long*& tk, int& id) {
                      const SceneD& S = t.s[RTSDF_FIND_SCENE(t, tri_off, gt)];
                      load_tri(verts + 3 * (int64_t)S.vert_off, S.V, tris + 3 * (int64_t)S.tri_off, gt - S.tri_off,
                               S.g, a, b, c);  // count > 0 implies valid
                      tri_range(a, b, c, S.g, r);
                      tnx = S.g.nx;
                      tny = S.g.ny;
                      tk = keys + S.vox_off;
                      id = gt - S.tri_off;
                  });
    }
}

// key -> (packed seed, representative triangle); voxels between scenes get EMPTY
__global__ void k_bvox_finalize(const __grid_constant__ BatchTable t, const unsigned long long* __restrict__ keys,
                                int64_t nvox, int32_t* __restrict__ seed, int32_t* __restrict__ rep) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const SceneD& S = t.s[RTSDF_FIND_SCENE(t, vox_off, v)];
    const int64_t lin = v - S.vox_off;
    const int64_t plane = (int64_t)S.g.nx * S.g.ny;
    if (lin >= plane * S.g.nz) {
        seed[v] = RTSDF_EMPTY;
        rep[v] = -1;
        return;
    }
    const unsigned long long key = __ldcs(keys + v);
    const bool empty = key == ~0ull;
    const int k = (int)(lin / plane), rem = (int)(lin - (int64_t)k * plane);
    const int j = rem / S.g.nx, i = rem - j * S.g.nx;
    seed[v] = empty ? RTSDF_EMPTY : pack_seed(i, j, k);
    rep[v] = empty ? -1 : (int32_t)(uint32_t)key;
}

// ------------------------------------------------------------------ BVH

__global__ void k_bbvh_headers(const __grid_constant__ BatchTable t, char* __restrict__ bvh) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= t.n) return;
    BvhHeader* h = reinterpret_cast<BvhHeader*>(bvh + t.s[s].bvh_off);
    h->n_leaves = 0;
    h->n_tris = t.s[s].T;
}

// key = (scene << 32) | Morton code: one sort orders every scene's triangles
// within the scene's own segment of the batch order
__global__ void k_bbvh_keys(const __grid_constant__ BatchTable t, const float* __restrict__ verts,
                            const int32_t* __restrict__ tris, int Ttot, unsigned long long* __restrict__ keys,
                            uint32_t* __restrict__ vals, char* __restrict__ bvh) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= Ttot) return;
    const int si = RTSDF_FIND_SCENE(t, tri_off, gt);
    const SceneD& S = t.s[si];
    const uint32_t code = tri_morton(verts + 3 * (int64_t)S.vert_off, S.V, tris + 3 * (int64_t)S.tri_off,
                                     gt - S.tri_off, S.g,
                                     reinterpret_cast<TriVox*>(bvh + S.bvh_off + bvh_tris_offset(S.T)));
    if (code != kInvalidKey) atomicAdd(&reinterpret_cast<BvhHeader*>(bvh + S.bvh_off)->n_leaves, 1);
    keys[gt] = ((unsigned long long)si << 32) | code;
    vals[gt] = (uint32_t)gt;
}

__device__ __forceinline__ BvhNode* scene_nodes(char* bvh, const SceneD& S) {
    return reinterpret_cast<BvhNode*>(bvh + S.bvh_off + bvh_nodes_offset());
}
__device__ __forceinline__ BvhLeaf* scene_leaves(char* bvh, const SceneD& S) {
    return reinterpret_cast<BvhLeaf*>(bvh + S.bvh_off + bvh_leaves_offset(S.T));
}

__global__ void k_bbvh_topology(const __grid_constant__ BatchTable t, const unsigned long long* __restrict__ keys,
                                char* __restrict__ bvh, int Ttot, int32_t* __restrict__ parent_inner,
                                int32_t* __restrict__ parent_leaf) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= Ttot) return;
    const SceneD& S = t.s[RTSDF_FIND_SCENE(t, tri_off, gi)];
    const int n = reinterpret_cast<const BvhHeader*>(bvh + S.bvh_off)->n_leaves;
    const int i = gi - S.tri_off;
    if (i >= n - 1) return;
    bvh_topology_node(keys + S.tri_off, n, i, scene_nodes(bvh, S), parent_inner + S.tri_off,
                      parent_leaf + S.tri_off);
}

__global__ void k_bbvh_leaves(const __grid_constant__ BatchTable t, const float* __restrict__ verts,
                              const int32_t* __restrict__ tris, const uint32_t* __restrict__ vals,
                              char* __restrict__ bvh, int Ttot, const int32_t* __restrict__ parent_inner,
                              const int32_t* __restrict__ parent_leaf, uint32_t* __restrict__ visits) {
    const int gj = blockIdx.x * blockDim.x + threadIdx.x;
    if (gj >= Ttot) return;
    const SceneD& S = t.s[RTSDF_FIND_SCENE(t, tri_off, gj)];
    const int n = reinterpret_cast<const BvhHeader*>(bvh + S.bvh_off)->n_leaves;
    const int j = gj - S.tri_off;
    if (j >= n) return;
    bvh_leaf_up(verts + 3 * (int64_t)S.vert_off, S.V, tris + 3 * (int64_t)S.tri_off, S.g, (int)vals[gj] - S.tri_off,
                j, n, scene_nodes(bvh, S), scene_leaves(bvh, S), parent_inner + S.tri_off, parent_leaf + S.tri_off,
                visits + S.tri_off);
}

// ------------------------------------------------------------------ jump flooding

struct PassD {
    const uint32_t* in;
    uint32_t* out;
    int32_t nx, ny, nz, k, chunk, nchunk, gbx, gby, block_start;
};

struct PassTable {
    int32_t n;
    PassD e[kMaxBatch];
};

__global__ void __launch_bounds__(kJX* kJY) k_bjfa_pass(const __grid_constant__ PassTable p) {
    const int b = blockIdx.x;
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.e[mid].block_start <= b) lo = mid; else hi = mid - 1;
    }
    const PassD& e = p.e[lo];
    const int local = b - e.block_start;
    jfa_column(e.in, e.out, e.nx, e.ny, e.nz, e.k, e.nchunk, e.chunk, local % e.gbx, (local / e.gbx) % e.gby,
               local / (e.gbx * e.gby));
}

// ------------------------------------------------------------------ coarse field + refine

// A scene's refinement arguments for bricks of BX x BY x BZ (built on the host into a
// RefineTable for each launch).
template <int BX, int BY, int BZ>
__host__ __device__ inline RefineArgs scene_args(const SceneD& S, const char* bvh, uint32_t frame, int accumulate) {
    RefineArgs a;
    a.g = S.g;
    a.tv = reinterpret_cast<const TriVox*>(bvh + S.bvh_off + bvh_tris_offset(S.T));
    a.T = S.T;
    a.mask2 = S.mask2;
    a.beta = S.beta;
    a.empty_dist = S.empty_dist;
    a.R = S.R;
    a.tmax = S.tmax;
    a.k0 = S.k0;
    a.k1 = S.k1;
    a.frame = frame;
    a.scene = S.scene;
    a.accumulate = accumulate;
    a.fallback = S.fallback;
    a.alpha = S.alpha;
    a.one_minus_alpha = 1.0f - S.alpha;
    a.ratio = 1;
    a.cnx = S.g.nx;
    a.cny = S.g.ny;
    a.cnz = S.g.nz;
    a.nbx = (S.g.nx + BX - 1) / BX;
    a.nby = (S.g.ny + BY - 1) / BY;
    a.nbz = (S.g.nz + BZ - 1) / BZ;
    a.per_ray = 0;
    return a;
}

// The refinement arguments of every scene for one launch (the brick shape, frame and
// accumulation mode of that launch), built on the host and passed as a grid-constant
// kernel parameter: the kernels read a scene's fields from the parameter bank with a
// warp-uniform index, as the single-scene kernels read their own RefineArgs, instead
// of assembling them in registers per brick.
struct RefineTable {
    RefineArgs a[kMaxBatch];
};

struct BatchGrids {
    const int32_t* buf_a;
    const int32_t* buf_b;
    const int32_t* rep_tri;
    uint32_t* dist_bits;
    uint32_t* front;
    uint32_t* back;
    float* sdf;
    const float* verts;
    const int32_t* tris;
    const char* bvh;
};

// both tables travel as kernel parameters (at most 32,764 bytes of them per launch)
static_assert(sizeof(BatchTable) + sizeof(RefineTable) + sizeof(BatchGrids) + 128 <= 32764, "kernel parameters");

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(512, 4) k_bresolve(const __grid_constant__ BatchTable t,
                                                  const __grid_constant__ RefineTable R, BatchGrids G,
                                                  unsigned long long* __restrict__ bmask,
                                                  int32_t* __restrict__ blist, uint32_t* __restrict__ count) {
    __shared__ unsigned long long smask[kMaxBricksPerTile];
    const int si = RTSDF_FIND_SCENE(t, tile_start, blockIdx.x);
    const SceneD& S = t.s[si];
    const int local = blockIdx.x - S.tile_start;
    const int gtx = (S.g.nx + 31) / 32, gty = (S.g.ny + 3) / 4;
    const int3 tb = make_int3(local % gtx, (local / gtx) % gty, local / (gtx * gty));
    const RefineArgs& a = R.a[si];
    const int64_t o = S.vox_off;
    resolve_tile<BX, BY, BZ>(a, tb, (S.flood_b ? G.buf_b : G.buf_a) + o, G.rep_tri + o, G.dist_bits + o, G.front + o,
                             G.back + o, G.sdf + o, bmask + S.brick_off, blist, count, nullptr, nullptr,
                             (int32_t)(si << kBrickBits), smask);
}

// Persistent, like k_refine: with kCull the bricks that refine_brick leaves to the
// per-ray launch go to dlist (as their work-list entries); with kRays the kernel is
// that launch and takes its bricks from dlist.
template <int BX, int BY, int BZ, int RPL, bool kCull, bool kRays = false>
__global__ void __launch_bounds__(kRefineMaxThreads, refine_warps_per_sm<RPL>() * 32 / kRefineMaxThreads) k_brefine(const __grid_constant__ BatchTable t,
                                                                  const __grid_constant__ RefineTable R, BatchGrids G,
                                                                  const char* __restrict__ bvh,
                                                                  const unsigned long long* __restrict__ bmask,
                                                                  const int32_t* __restrict__ blist,
                                                                  int32_t* __restrict__ dlist,
                                                                  uint32_t* __restrict__ count,
                                                                  rtsdf_counters* counters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmemT<RPL>& w = reinterpret_cast<WarpSmemT<RPL>*>(smem_raw)[warp];
    const uint32_t nact = count[kRays ? 3 : 0];
    uint32_t n_hit = 0, n_fail = 0, n_ovf = 0;
    while (true) {
        uint32_t wk = 0;
        if (lane == 0) wk = atomicAdd(count + (kRays ? 4 : 1), 1u);
        wk = __shfl_sync(0xffffffffu, wk, 0);
        if (wk >= nact) break;
        const uint32_t e = (uint32_t)(kRays ? dlist[wk] : blist[wk]);
        const int si = (int)(e >> kBrickBits), b = (int)(e & ((1u << kBrickBits) - 1u));
        const SceneD& S = t.s[si];
        const RefineArgs& a = R.a[si];
        const BvhHeader* hdr = reinterpret_cast<const BvhHeader*>(bvh + S.bvh_off);
        const BvhNode* nodes = reinterpret_cast<const BvhNode*>(bvh + S.bvh_off + bvh_nodes_offset());
        const BvhLeaf* leaves = reinterpret_cast<const BvhLeaf*>(bvh + S.bvh_off + bvh_leaves_offset(S.T));
        const int n_leaves = hdr->n_leaves;
        const int n_inner = n_leaves > 1 ? n_leaves - 1 : 1;
        const int bx = b % a.nbx, by = (b / a.nbx) % a.nby, bz = b / (a.nbx * a.nby);
        const int64_t o = S.vox_off;
        const bool deferred = refine_brick<BX, BY, BZ, false, RPL, false, kCull, kRays>(
            a, nodes, leaves, n_leaves, n_inner, (S.flood_b ? G.buf_b : G.buf_a) + o, G.rep_tri + o,
            bmask[S.brick_off + b], bx, by, bz, G.dist_bits + o, G.front + o, G.back + o, G.sdf + o, nullptr, nullptr,
            w, n_hit, n_fail, n_ovf);
        if (deferred && lane == 0) dlist[atomicAdd(count + 3, 1u)] = (int32_t)e;
    }
    if (counters) {
        if (n_hit) atomicAdd(&counters->rays_hit, n_hit);
        if (n_fail) atomicAdd(&counters->rays_failed, n_fail);
    }
    if (lane == 0 && n_ovf) atomicAdd(count + 2, n_ovf);
}

__global__ void k_brefine_report(const uint32_t* __restrict__ count, const unsigned long long* __restrict__ bmask,
                                 int64_t nb, rtsdf_counters* counters) {
    uint32_t n = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        n += __popcll(bmask[b]);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&counters->masked_voxels, n);
    if (blockIdx.x == 0 && threadIdx.x == 0 && count[2]) atomicAdd(&counters->stack_overflow, count[2]);
}

// ------------------------------------------------------------------ the shapes the refinement is built for

struct Shape {
    int bx, by, bz;
};
constexpr Shape kShapes[] = {{4, 4, 4}, {8, 4, 2}, {16, 2, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

static int64_t shape_bricks(const rtsdf_grid& g, const Shape& sh) {
    return (int64_t)((g.nx + sh.bx - 1) / sh.bx) * ((g.ny + sh.by - 1) / sh.by) * ((g.nz + sh.bz - 1) / sh.bz);
}

}  // namespace rtsdf

using namespace rtsdf;

// ------------------------------------------------------------------ the plan (host)

struct rtsdf_batch_plan {
    std::vector<rtsdf_batch_scene> scenes;
    std::vector<rtsdf_batch_layout> layout;
    int32_t S = 0;
    int64_t nvox = 0;
    int32_t Vtot = 0, Ttot = 0;
    int32_t ntiles = 0;
    int64_t max_bricks = 0;
    size_t bvh_bytes = 0;
    int32_t npasses = 0;
    rtsdf_batch_tuning tuning{4, 4, 4, 2, 1};
    // workspace layout (byte offsets)
    size_t off_keys = 0, off_counts = 0, off_offsets = 0, off_scan = 0;
    size_t off_k64a = 0, off_k64b = 0, off_va = 0, off_vb = 0, off_sort = 0, off_pin = 0, off_pl = 0, off_vis = 0;
    size_t off_count = 0, off_bmask = 0, off_blist = 0, off_dlist = 0, ws_bytes = 0;
    // the captured JFA chain
    cudaGraphExec_t jfa_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    const void* graph_a = nullptr;
    const void* graph_b = nullptr;
    int graph_device = -1;
};

namespace {

bool grid_valid(const rtsdf_grid& g) {
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > RTSDF_MAX_DIM || g.ny > RTSDF_MAX_DIM || g.nz > RTSDF_MAX_DIM)
        return false;
    if (!(g.h > 0.0f) || !isfinite(g.h)) return false;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(g.origin[a])) return false;
    return true;
}

bool tuning_valid(const rtsdf_batch_tuning& t) {
    bool shape = false;
    for (int i = 0; i < kNumShapes; ++i)
        shape |= kShapes[i].bx == t.brick_x && kShapes[i].by == t.brick_y && kShapes[i].bz == t.brick_z;
    return shape && (t.warps_per_cta == 1 || t.warps_per_cta == 2 || t.warps_per_cta == 4) &&
           (t.use_graph == 0 || t.use_graph == 1);
}

BatchTable make_table(const rtsdf_batch_plan& P, const Shape& sh) {
    BatchTable t;
    memset(&t, 0, sizeof(t));
    t.n = P.S;
    t.nbx_div = sh.bx;
    t.nby_div = sh.by;
    t.nbz_div = sh.bz;
    int64_t brick = 0;
    int32_t tile = 0;
    for (int s = 0; s < P.S; ++s) {
        const rtsdf_batch_scene& sc = P.scenes[s];
        const rtsdf_batch_layout& L = P.layout[s];
        SceneD& d = t.s[s];
        d.g = to_dev(sc.grid);
        d.V = sc.V;
        d.T = sc.T;
        d.vert_off = L.vertex_offset;
        d.tri_off = L.triangle_offset;
        d.vox_off = L.voxel_offset;
        d.bvh_off = L.bvh_offset;
        d.brick_off = brick;
        brick += shape_bricks(sc.grid, sh);
        d.tile_start = tile;
        tile += ((sc.grid.nx + 31) / 32) * ((sc.grid.ny + 3) / 4) * ((sc.grid.nz + 3) / 4);
        d.flood_b = L.flooded_in_b;
        d.mask2 = sc.refine.mask_vox * sc.refine.mask_vox;
        d.beta = sc.refine.beta_vox;
        d.empty_dist = (float)(sc.grid.nx + sc.grid.ny + sc.grid.nz);
        d.tmax = sc.refine.max_ray_vox;
        d.alpha = sc.refine.decay_alpha;
        d.R = sc.refine.rays_per_voxel;
        d.fallback = sc.refine.sign_fallback;
        d.k0 = sc.refine.key[0];
        d.k1 = sc.refine.key[1];
        d.scene = sc.refine.scene_id;
    }
    return t;
}

cudaStream_t cs(rtsdf_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// The JFA passes of the batch: pass p runs, for every scene with nsteps >= P - p,
// its step number nsteps - (P - p), reading the buffer its previous pass wrote.
rtsdf_status enqueue_jfa(const rtsdf_batch_plan& P, uint32_t* a, uint32_t* b, cudaStream_t s) {
    for (int p = 0; p < P.npasses; ++p) {
        PassTable pt;
        memset(&pt, 0, sizeof(pt));
        int32_t blocks = 0;
        for (int si = 0; si < P.S; ++si) {
            const rtsdf_batch_scene& sc = P.scenes[si];
            const int first = P.npasses - sc.nsteps;  // the scene's first pass
            if (p < first) continue;
            const int idx = p - first;
            const int64_t o = P.layout[si].voxel_offset;
            const bool from_a = (idx % 2) == 0;
            PassD& e = pt.e[pt.n++];
            e.in = (from_a ? a : b) + o;
            e.out = (from_a ? b : a) + o;
            e.nx = sc.grid.nx;
            e.ny = sc.grid.ny;
            e.nz = sc.grid.nz;
            e.k = sc.steps[idx];
            // the single-scene rule: 32-plane chunks for grids of 16 M voxels and more, else 16
            e.chunk = (int64_t)e.nx * e.ny * e.nz >= (int64_t)(16 << 20) ? kChunk : kChunkSmall;
            const int nq = (e.nz + e.k - 1) / e.k;
            e.nchunk = (nq + e.chunk - 1) / e.chunk;
            e.gbx = jfa_xblocks(e.nx, e.k);
            e.gby = (e.ny + kJY - 1) / kJY;
            e.block_start = blocks;
            blocks += e.gbx * e.gby * e.k * e.nchunk;
        }
        if (pt.n == 0) continue;
        k_bjfa_pass<<<blocks, dim3(kJX, kJY, 1), 0, s>>>(pt);
        RTSDF_LAUNCHED();
    }
    return RTSDF_OK;
}

rtsdf_status run_jfa(rtsdf_batch_plan& P, uint32_t* a, uint32_t* b, cudaStream_t s) {
    if (!P.tuning.use_graph) return enqueue_jfa(P, a, b, s);
    int dev = -1;
    RTSDF_CUDA(cudaGetDevice(&dev));
    if (!P.jfa_exec || P.graph_a != a || P.graph_b != b || P.graph_device != dev) {
        if (P.jfa_exec) {
            cudaGraphExecDestroy(P.jfa_exec);
            P.jfa_exec = nullptr;
        }
        if (P.capture_stream && P.graph_device != dev) {
            cudaStreamDestroy(P.capture_stream);
            P.capture_stream = nullptr;
        }
        if (!P.capture_stream) RTSDF_CUDA(cudaStreamCreateWithFlags(&P.capture_stream, cudaStreamNonBlocking));
        RTSDF_CUDA(cudaStreamBeginCapture(P.capture_stream, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = launches();
        const rtsdf_status st = enqueue_jfa(P, a, b, P.capture_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(P.capture_stream, &graph);
        note_launch(-(int)(launches() - before));  // captured, not launched
        if (st != RTSDF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess) return RTSDF_ECUDA;
        const cudaError_t ie = cudaGraphInstantiate(&P.jfa_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            P.jfa_exec = nullptr;
            return RTSDF_ECUDA;
        }
        P.graph_a = a;
        P.graph_b = b;
        P.graph_device = dev;
    }
    RTSDF_CUDA(cudaGraphLaunch(P.jfa_exec, s));
    note_launch(P.npasses);
    return RTSDF_OK;
}

template <int BX, int BY, int BZ, int RPL, bool kCull>
rtsdf_status launch_refine(const rtsdf_batch_plan& P, const rtsdf_batch_buffers& B, uint32_t frame, int accumulate,
                           rtsdf_counters* counters, int warps, cudaStream_t s) {
    const Shape sh{BX, BY, BZ};
    const BatchTable t = make_table(P, sh);
    RefineTable R;
    memset(&R, 0, sizeof(R));
    for (int si = 0; si < t.n; ++si) {
        R.a[si] = scene_args<BX, BY, BZ>(t.s[si], static_cast<const char*>(B.bvh), frame, accumulate);
        // coarse scenes trace the rays of their overflowing bricks one by one
        const rtsdf_batch_scene& sc = P.scenes[si];
        R.a[si].per_ray = kCull && staged_estimate(sc.T, sc.grid.nx, sc.grid.ny, sc.grid.nz, sc.refine.max_ray_vox,
                                                   BX, BY, BZ) >= per_ray_estimate(sc.refine.rays_per_voxel);
    }
    char* ws = static_cast<char*>(B.ws);
    auto* count = reinterpret_cast<uint32_t*>(ws + P.off_count);
    auto* bmask = reinterpret_cast<unsigned long long*>(ws + P.off_bmask);
    auto* blist = reinterpret_cast<int32_t*>(ws + P.off_blist);
    auto* dlist = reinterpret_cast<int32_t*>(ws + P.off_dlist);
    bool per_ray = false;
    for (int si = 0; si < t.n; ++si) per_ray = per_ray || R.a[si].per_ray != 0;
    BatchGrids G{B.seed, B.buf_b, B.rep_tri, B.dist_bits, B.front, B.back, B.sdf, B.verts, B.tris,
                 static_cast<const char*>(B.bvh)};
    RTSDF_CUDA(cudaMemsetAsync(count, 0, 32, s));
    k_bresolve<BX, BY, BZ><<<P.ntiles, 512, 0, s>>>(t, R, G, bmask, blist, count);
    RTSDF_LAUNCHED();
    const size_t smem = sizeof(WarpSmemT<RPL>) * (size_t)warps;
    static bool attr_set[64] = {false};
    int dev = 0;
    RTSDF_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RTSDF_CUDA(cudaFuncSetAttribute(k_brefine<BX, BY, BZ, RPL, kCull>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(WarpSmemT<RPL>) * 4)));
        if constexpr (kCull)
            RTSDF_CUDA(cudaFuncSetAttribute(k_brefine<BX, BY, BZ, RPL, kCull, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sizeof(WarpSmemT<RPL>) * 4)));
        attr_set[dev] = true;
    }
    // the same resident warps per SM for every CTA size (shared memory bound)
    const int ctas = num_sms() * (refine_warps_per_sm<RPL>() / warps);
    k_brefine<BX, BY, BZ, RPL, kCull><<<ctas, 32 * warps, smem, s>>>(t, R, G, static_cast<const char*>(B.bvh), bmask,
                                                                     blist, dlist, count, counters);
    RTSDF_LAUNCHED();
    if constexpr (kCull) {
        if (per_ray) {  // the bricks the first launch left to the per-ray walk
            k_brefine<BX, BY, BZ, RPL, kCull, true><<<ctas, 32 * warps, smem, s>>>(
                t, R, G, static_cast<const char*>(B.bvh), bmask, blist, dlist, count, counters);
            RTSDF_LAUNCHED();
        }
    }
    if (counters) {
        int64_t nb = 0;
        for (int si = 0; si < P.S; ++si) nb += shape_bricks(P.scenes[si].grid, sh);
        k_brefine_report<<<num_sms(), 256, 0, s>>>(count, bmask, nb, counters);
        RTSDF_LAUNCHED();
    }
    return RTSDF_OK;
}

rtsdf_status refine_step(const rtsdf_batch_plan& P, const rtsdf_batch_buffers& B, uint32_t frame, int accumulate,
                         rtsdf_counters* counters, const rtsdf_batch_tuning& tu, cudaStream_t s) {
    const int w = tu.warps_per_cta;
    int rmax = 1;  // one ray group per brick for up to rpl rays (the largest ray count of the batch)
    for (const rtsdf_batch_scene& sc : P.scenes) rmax = sc.refine.rays_per_voxel > rmax ? sc.refine.rays_per_voxel : rmax;
    const int rpl = rmax <= 2 ? 2 : (rmax <= 4 ? 4 : (rmax <= 8 ? 8 : 16));
    // the culling instantiation when some scene is coarse (many triangles within a brick's reach)
    bool cull = false;
    for (const rtsdf_batch_scene& sc : P.scenes)
        cull = cull || staged_estimate(sc.T, sc.grid.nx, sc.grid.ny, sc.grid.nz, sc.refine.max_ray_vox, tu.brick_x,
                                       tu.brick_y, tu.brick_z) >= kCullEstimate;
#define RTSDF_BATCH_CASE(X, Y, Z, R)                                                                  \
    if (tu.brick_x == X && rpl == R)                                                                  \
        return cull ? launch_refine<X, Y, Z, R, true>(P, B, frame, accumulate, counters, w, s)        \
                    : launch_refine<X, Y, Z, R, false>(P, B, frame, accumulate, counters, w, s);
    RTSDF_BATCH_CASE(4, 4, 4, 2) RTSDF_BATCH_CASE(4, 4, 4, 4) RTSDF_BATCH_CASE(4, 4, 4, 8)
    RTSDF_BATCH_CASE(4, 4, 4, 16)
    RTSDF_BATCH_CASE(8, 4, 2, 2) RTSDF_BATCH_CASE(8, 4, 2, 4) RTSDF_BATCH_CASE(8, 4, 2, 8)
    RTSDF_BATCH_CASE(8, 4, 2, 16)
    RTSDF_BATCH_CASE(16, 2, 2, 2) RTSDF_BATCH_CASE(16, 2, 2, 4) RTSDF_BATCH_CASE(16, 2, 2, 8)
    RTSDF_BATCH_CASE(16, 2, 2, 16)
#undef RTSDF_BATCH_CASE
    return RTSDF_EINVAL;
}

rtsdf_status buffers_ok(const rtsdf_batch_plan* P, const rtsdf_batch_buffers* b) {
    if (!P || !b) return RTSDF_EINVAL;
    auto al = [](const void* p, size_t a) { return p != nullptr && reinterpret_cast<uintptr_t>(p) % a == 0; };
    if ((P->Ttot > 0 && (!al(b->verts, 4) || !al(b->tris, 4))) || !al(b->seed, 16) || !al(b->buf_b, 16) ||
        !al(b->rep_tri, 16) || !al(b->bvh, 256) || !al(b->dist_bits, 16) || !al(b->front, 16) || !al(b->back, 16) ||
        !al(b->sdf, 16) || !al(b->ws, 256) || b->seed == b->buf_b)
        return RTSDF_EINVAL;
    if (b->bvh_bytes < P->bvh_bytes || b->ws_bytes < P->ws_bytes) return RTSDF_ENOMEM;
    return RTSDF_OK;
}

rtsdf_status rebuild(rtsdf_batch_plan& P, const rtsdf_batch_buffers& B, uint32_t frame, int accumulate,
                     rtsdf_counters* counters, cudaStream_t s) {
    const Shape sh{P.tuning.brick_x, P.tuning.brick_y, P.tuning.brick_z};
    const BatchTable t = make_table(P, sh);
    char* ws = static_cast<char*>(B.ws);
    char* bvh = static_cast<char*>(B.bvh);
    // voxelize
    auto* keys = reinterpret_cast<unsigned long long*>(ws + P.off_keys);
    auto* counts = reinterpret_cast<uint32_t*>(ws + P.off_counts);
    auto* offsets = reinterpret_cast<uint64_t*>(ws + P.off_offsets);
    RTSDF_CUDA(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * (size_t)P.nvox, s));
    if (P.Ttot > 0) {
        k_bvox_count<<<(P.Ttot + 255) / 256, 256, 0, s>>>(t, B.verts, B.tris, P.Ttot, counts, counters);
        RTSDF_LAUNCHED();
        RTSDF_TRY(scan_u32_to_u64(counts, offsets, (size_t)P.Ttot, ws + P.off_scan, s));
        k_bvox_test<<<num_sms() * 8, 256, 0, s>>>(t, B.verts, B.tris, P.Ttot, offsets, keys);
        RTSDF_LAUNCHED();
    }
    k_bvox_finalize<<<(unsigned)((P.nvox + 255) / 256), 256, 0, s>>>(t, keys, P.nvox, B.seed, B.rep_tri);
    RTSDF_LAUNCHED();
    // BVH
    k_bbvh_headers<<<1, kMaxBatch, 0, s>>>(t, bvh);
    RTSDF_LAUNCHED();
    if (P.Ttot > 0) {
        auto* ka = reinterpret_cast<unsigned long long*>(ws + P.off_k64a);
        auto* kb = reinterpret_cast<unsigned long long*>(ws + P.off_k64b);
        auto* va = reinterpret_cast<uint32_t*>(ws + P.off_va);
        auto* vb = reinterpret_cast<uint32_t*>(ws + P.off_vb);
        auto* pin = reinterpret_cast<int32_t*>(ws + P.off_pin);
        auto* pl = reinterpret_cast<int32_t*>(ws + P.off_pl);
        auto* vis = reinterpret_cast<uint32_t*>(ws + P.off_vis);
        k_bbvh_keys<<<(P.Ttot + 255) / 256, 256, 0, s>>>(t, B.verts, B.tris, P.Ttot, ka, va, bvh);
        RTSDF_LAUNCHED();
        int scene_bits = 0;
        while ((1 << scene_bits) < P.S) ++scene_bits;
        unsigned long long* sk = nullptr;
        uint32_t* sv = nullptr;
        RTSDF_TRY(radix_sort_pairs<unsigned long long>(ka, va, kb, vb, P.Ttot, 32 + scene_bits, ws + P.off_sort, s,
                                                       &sk, &sv));
        RTSDF_CUDA(cudaMemsetAsync(vis, 0, sizeof(uint32_t) * (size_t)P.Ttot, s));
        k_bbvh_topology<<<(P.Ttot + 255) / 256, 256, 0, s>>>(t, sk, bvh, P.Ttot, pin, pl);
        RTSDF_LAUNCHED();
        k_bbvh_leaves<<<(P.Ttot + 255) / 256, 256, 0, s>>>(t, B.verts, B.tris, sv, bvh, P.Ttot, pin, pl, vis);
        RTSDF_LAUNCHED();
    }
    // jump flooding
    RTSDF_TRY(run_jfa(P, reinterpret_cast<uint32_t*>(B.seed), reinterpret_cast<uint32_t*>(B.buf_b), s));
    // coarse field, ray mask, refinement
    return refine_step(P, B, frame, accumulate, counters, P.tuning, s);
}

}  // namespace

extern "C" {

rtsdf_status rtsdf_batch_plan_create(const rtsdf_batch_scene* scenes, int32_t S, rtsdf_batch_plan** plan) {
    if (!plan) return RTSDF_EINVAL;
    *plan = nullptr;
    if (!scenes || S < 1 || S > kMaxBatch) return RTSDF_EINVAL;
    int64_t vox = 0, V = 0, T = 0, tiles = 0;
    size_t bvh = 0;
    int32_t npasses = 0;
    for (int s = 0; s < S; ++s) {
        const rtsdf_batch_scene& sc = scenes[s];
        if (!grid_valid(sc.grid) || sc.V < 0 || sc.T < 0 || sc.nsteps < 0 || sc.nsteps > RTSDF_BATCH_MAX_STEPS)
            return RTSDF_EINVAL;
        for (int i = 0; i < sc.nsteps; ++i)
            if (sc.steps[i] < 1 || sc.steps[i] > RTSDF_MAX_DIM) return RTSDF_EINVAL;
        const rtsdf_refine_params& r = sc.refine;
        if (r.rays_per_voxel < 1 || r.rays_per_voxel > 4096 || !(r.mask_vox >= 0.0f) || !isfinite(r.mask_vox) ||
            !(r.max_ray_vox > 0.0f) || !isfinite(r.beta_vox))
            return RTSDF_EINVAL;
        V += sc.V;
        T += sc.T;
        vox += ((int64_t)sc.grid.nx * sc.grid.ny * sc.grid.nz + 63) / 64 * 64;
        tiles += (int64_t)((sc.grid.nx + 31) / 32) * ((sc.grid.ny + 3) / 4) * ((sc.grid.nz + 3) / 4);
        bvh += align_up(bvh_bytes(sc.T), 256);
        if (sc.nsteps > npasses) npasses = sc.nsteps;
    }
    if (V > (1 << 28) || T > (1 << 28) || tiles > (1 << 30)) return RTSDF_EINVAL;
    for (int s = 0; s < S; ++s) {  // brick indices must fit the work-list entry
        for (int i = 0; i < kNumShapes; ++i)
            if (shape_bricks(scenes[s].grid, kShapes[i]) >= (1 << kBrickBits)) return RTSDF_EINVAL;
    }
    rtsdf_batch_plan* P = new (std::nothrow) rtsdf_batch_plan();
    if (!P) return RTSDF_ENOMEM;
    try {
        P->scenes.assign(scenes, scenes + S);
        P->layout.resize(S);
    } catch (...) {
        delete P;
        return RTSDF_ENOMEM;
    }
    P->S = S;
    P->nvox = vox;
    P->Vtot = (int32_t)V;
    P->Ttot = (int32_t)T;
    P->ntiles = (int32_t)tiles;
    P->bvh_bytes = bvh;
    P->npasses = npasses;
    int64_t vo = 0;
    int32_t vv = 0, tt = 0;
    size_t bo = 0;
    for (int s = 0; s < S; ++s) {
        const rtsdf_batch_scene& sc = scenes[s];
        rtsdf_batch_layout& L = P->layout[s];
        L.voxel_offset = vo;
        L.vertex_offset = vv;
        L.triangle_offset = tt;
        L.bvh_offset = (int64_t)bo;
        L.flooded_in_b = sc.nsteps % 2;
        L.reserved = 0;
        vo += ((int64_t)sc.grid.nx * sc.grid.ny * sc.grid.nz + 63) / 64 * 64;
        vv += sc.V;
        tt += sc.T;
        bo += align_up(bvh_bytes(sc.T), 256);
    }
    int64_t mb = 0;
    for (int i = 0; i < kNumShapes; ++i) {
        int64_t nb = 0;
        for (int s = 0; s < S; ++s) nb += shape_bricks(scenes[s].grid, kShapes[i]);
        if (nb > mb) mb = nb;
    }
    P->max_bricks = mb;
    const size_t n = (size_t)(T > 0 ? T : 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, 256);
        return o;
    };
    P->off_keys = take(8 * (size_t)vox);
    P->off_counts = take(4 * n);
    P->off_offsets = take(8 * (n + 1));
    P->off_scan = take(scan_u32_to_u64_scratch(n));
    P->off_k64a = take(8 * n);
    P->off_k64b = take(8 * n);
    P->off_va = take(4 * n);
    P->off_vb = take(4 * n);
    P->off_sort = take(radix_sort_scratch<unsigned long long>((int)n));
    P->off_pin = take(4 * n);
    P->off_pl = take(4 * n);
    P->off_vis = take(4 * n);
    P->off_count = take(64);
    P->off_bmask = take(8 * (size_t)mb);
    P->off_blist = take(4 * (size_t)mb);
    P->off_dlist = take(4 * (size_t)mb);
    P->ws_bytes = off;
    *plan = P;
    return RTSDF_OK;
}

void rtsdf_batch_plan_destroy(rtsdf_batch_plan* plan) {
    if (!plan) return;
    if (plan->jfa_exec) cudaGraphExecDestroy(plan->jfa_exec);
    if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
    delete plan;
}

rtsdf_status rtsdf_batch_layout_of(const rtsdf_batch_plan* plan, int32_t scene, rtsdf_batch_layout* out) {
    if (!plan || !out || scene < 0 || scene >= plan->S) return RTSDF_EINVAL;
    *out = plan->layout[scene];
    return RTSDF_OK;
}

size_t rtsdf_batch_voxels(const rtsdf_batch_plan* plan) { return plan ? (size_t)plan->nvox : 0; }
size_t rtsdf_batch_bvh_bytes(const rtsdf_batch_plan* plan) { return plan ? plan->bvh_bytes : 0; }
size_t rtsdf_batch_workspace(const rtsdf_batch_plan* plan) { return plan ? plan->ws_bytes : 0; }

rtsdf_status rtsdf_batch_get_tuning(const rtsdf_batch_plan* plan, rtsdf_batch_tuning* out) {
    if (!plan || !out) return RTSDF_EINVAL;
    *out = plan->tuning;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_set_tuning(rtsdf_batch_plan* plan, const rtsdf_batch_tuning* t) {
    if (!plan || !t || !tuning_valid(*t)) return RTSDF_EINVAL;
    plan->tuning = *t;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_rebuild(rtsdf_batch_plan* plan, const rtsdf_batch_buffers* b, uint32_t frame_index,
                                 int32_t accumulate, rtsdf_counters* counters, rtsdf_stream stream) {
    RTSDF_TRY(buffers_ok(plan, b));
    if (counters && reinterpret_cast<uintptr_t>(counters) % 8) return RTSDF_EINVAL;
    if (accumulate < 0 || accumulate > 2) return RTSDF_EINVAL;
    if (accumulate == 2)
        for (const rtsdf_batch_scene& sc : plan->scenes)
            if (!(sc.refine.decay_alpha >= 0.0f && sc.refine.decay_alpha <= 1.0f)) return RTSDF_EINVAL;
    return rebuild(*plan, *b, frame_index, accumulate, counters, cs(stream));
}

rtsdf_status rtsdf_batch_autotune(rtsdf_batch_plan* plan, const rtsdf_batch_buffers* b, int32_t reps,
                                  float* best_ms, rtsdf_stream stream) {
    RTSDF_TRY(buffers_ok(plan, b));
    if (reps < 1 || reps > 1000) return RTSDF_EINVAL;
    const cudaStream_t s = cs(stream);
    RTSDF_TRY(rebuild(*plan, *b, 0, 0, nullptr, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RTSDF_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return RTSDF_ECUDA;
    }
    rtsdf_status st = RTSDF_OK;
    float best = -1.0f;
    rtsdf_batch_tuning best_t = plan->tuning;
    const int warps[3] = {1, 2, 4};
    for (int i = 0; i < kNumShapes && st == RTSDF_OK; ++i) {
        for (int w = 0; w < 3 && st == RTSDF_OK; ++w) {
            rtsdf_batch_tuning tu = plan->tuning;
            tu.brick_x = kShapes[i].bx;
            tu.brick_y = kShapes[i].by;
            tu.brick_z = kShapes[i].bz;
            tu.warps_per_cta = warps[w];
            st = refine_step(*plan, *b, 0, 0, nullptr, tu, s);  // warm-up
            if (cudaEventRecord(e0, s) != cudaSuccess) st = RTSDF_ECUDA;
            for (int r = 0; r < reps && st == RTSDF_OK; ++r) st = refine_step(*plan, *b, 0, 0, nullptr, tu, s);
            if (st == RTSDF_OK && cudaEventRecord(e1, s) != cudaSuccess) st = RTSDF_ECUDA;
            float ms = 0.0f;
            if (st == RTSDF_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                                   cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = RTSDF_ECUDA;
            ms /= (float)reps;
            if (st == RTSDF_OK && (best < 0.0f || ms < best)) {
                best = ms;
                best_t = tu;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RTSDF_OK) return st;
    plan->tuning = best_t;
    if (best_ms) *best_ms = best;
    return RTSDF_OK;
}

}  // extern "C"
