// The per-tile and per-brick bodies of the coarse field / ray mask pass and of
// the ray-sampled refinement (Sec. 2.1-2.3), shared by the single-scene kernels
// (refine.cu) and the batched ones (batch.cu).  Templated on the brick shape
// BX x BY x BZ (64 voxels, one bit each in a 64-bit mask): the resolve tile is
// 32 x 4 x 4 voxels, so BX divides 32 and BY, BZ divide 4.
#pragma once

#include <float.h>

#include "rtsdf_device.cuh"

namespace rtsdf {

constexpr int kListCap = 256;        // staged leaves per warp and round
constexpr int kStackCapW = 256;      // traversal stack per warp (entries)
constexpr int kNarrowMargin = 96;    // > depth of any tree the builder makes (30-bit codes + 32 index bits)
constexpr int kRaysPerLane = 8;      // rays of a voxel per group for up to 8 rays (one lane per voxel)
constexpr int kCullMinStaged = 160;  // staged triangles from which a brick culls (voxel, chunk) combinations
constexpr double kCullEstimate = 150.0;  // staged_estimate from which a launch takes the culling instantiation

// Triangles a brick of BX x BY x BZ voxels would stage if the mesh filled the grid
// evenly: T times the fraction of the grid its reach box (grown by the ray length)
// covers.  A coarse grid, whose ray length spans much of the scene, scores in the
// hundreds or thousands (the 400x200x400 room: 27; a 32^3 grid with 50 k triangles:
// 12 k).  Launches above kCullEstimate take the instantiation that culls (voxel,
// chunk) combinations (chunk_voxels); the others keep the plain loop, whose code
// runs faster when no brick stages that many triangles.
inline double staged_estimate(int T, int nx, int ny, int nz, float tmax, int bx, int by, int bz) {
    const double e = 2.0 * (double)tmax;
    const double f = ((double)bx + e) * ((double)by + e) * ((double)bz + e) / ((double)nx * ny * nz);
    return (double)T * (f < 1.0 ? f : 1.0);
}
// Staged-triangle estimate from which a launch (or a batch's scene) with R rays per
// voxel traces the rays of its overflowing bricks through the BVH one by one
// (ray_closest) instead of staging: the staged path costs about the same per staged
// triangle whatever R, the per-ray walk a fixed amount per ray, so the crossover grows
// with R (measured on the room at 128x64x128: 1 ray 3.0 -> 0.58 ms, 5 rays 3.65 ->
// 2.36 ms, 10 rays 4.5 -> 6.0 ms, at an estimate of 830).
inline double per_ray_estimate(int R) { return 150.0 + 100.0 * (double)(R > 1 ? R - 1 : 0); }
constexpr int kRefineMaxThreads = 128;                // refine CTAs hold 1, 2 or 4 warps
constexpr int kRefineWarpsPerSm = 20;                 // resident refine warps per SM (shared memory bound)
constexpr int kRefineWarpsPerSm16 = 12;               // the same with 16-ray groups (twice the ray rows)

template <int BX, int BY, int BZ>
struct BrickShape {
    static_assert(BX * BY * BZ == 64 || BX * BY * BZ == 32, "a brick holds 64 or 32 voxels");
    static_assert(32 % BX == 0 && 4 % BY == 0 && 4 % BZ == 0, "bricks tile the 32x4x4 resolve tile");
    static constexpr int kPerTile = (32 / BX) * (4 / BY) * (4 / BZ);  // 8 or 16
};

struct RefineArgs {
    GridD g;
    int T;
    const TriVox* tv;  // the BVH's voxel-space triangle table (vertices in voxel units)
    float mask2;
    float beta;
    float empty_dist;
    int R;
    float tmax;
    uint32_t k0, k1, frame, scene;
    int accumulate, fallback;
    float alpha, one_minus_alpha;  // Eq. (1) decay (accumulate = 2)
    int nbx, nby, nbz;  // brick grid
    int ratio;          // fine voxels per coarse voxel along each axis (1: one grid)
    int cnx, cny, cnz;  // coarse grid of the flooded seeds and representative triangles
    int per_ray;        // culling instantiation: overflowing bricks go to the per-ray launch
};

constexpr int kMaxBricksPerTile = 16;

// Index of the coarse voxel holding fine voxel (i, j, k) (the two-resolution form of
// Sec. 2.5.1: flooded seeds and representative triangles live on the coarse grid).
__device__ __forceinline__ int64_t coarse_index(const RefineArgs& a, int i, int j, int k, int& ic, int& jc, int& kc) {
    ic = a.ratio == 1 ? i : i / a.ratio;
    jc = a.ratio == 1 ? j : j / a.ratio;
    kc = a.ratio == 1 ? k : k / a.ratio;
    return ((int64_t)kc * a.cny + jc) * a.cnx + ic;
}

// One 32x4x4 tile of voxels (512 threads, tile coordinates tb): coarse distance u_c
// to the representative triangle of the flooded seed (with two resolutions: the
// seed of the coarse voxel holding the fine voxel; the mask compares the integer
// seed distance in coarse voxels); unmasked voxels get their
// final value (u_c - beta) and the state (u_c, 0, 0); masked voxels initialise their
// refine state (and, when tracked, the coarse source takes the winner record where
// it sets the distance).
// The tile's bricks get 64-bit masks of their masked voxels from warp ballots, and
// bricks with any masked voxel are appended to the work list as (tag | brick).
template <int BX, int BY, int BZ>
__device__ __forceinline__ void resolve_tile(const RefineArgs& a, int3 tb, const int32_t* __restrict__ nearest,
                                             const int32_t* __restrict__ rep_tri, uint32_t* __restrict__ dist_bits,
                                             uint32_t* __restrict__ front, uint32_t* __restrict__ back,
                                             float* __restrict__ sdf, unsigned long long* __restrict__ bmask,
                                             int32_t* __restrict__ blist, uint32_t* __restrict__ count,
                                             uint32_t* __restrict__ win_ray, int32_t* __restrict__ win_tri,
                                             int32_t tag, unsigned long long* smask) {
    constexpr int kBpx = 32 / BX, kBpy = 4 / BY, kPer = BrickShape<BX, BY, BZ>::kPerTile;
    const int tx = threadIdx.x & 31, ty = (threadIdx.x >> 5) & 3, tz = threadIdx.x >> 7;
    const int i = tb.x * 32 + tx, j = tb.y * 4 + ty, k = tb.z * 4 + tz;
    if (threadIdx.x < kPer) smask[threadIdx.x] = 0ull;
    __syncthreads();
    bool masked = false;
    if (i < a.g.nx && j < a.g.ny && k < a.g.nz) {
        const int64_t lin = ((int64_t)k * a.g.ny + j) * a.g.nx + i;
        int ic, jc, kc;
        const int32_t s = __ldg(nearest + coarse_index(a, i, j, k, ic, jc, kc));
        int32_t rep = -1;
        int si = 0, sj = 0, sk = 0;
        if (s != RTSDF_EMPTY) {
            si = s & 1023;
            sj = (s >> 10) & 1023;
            sk = (s >> 20) & 1023;
            rep = __ldg(rep_tri + ((int64_t)sk * a.cny + sj) * a.cnx + si);
        }
        float uc = a.empty_dist;
        float3 A, B, C;
        if (rep >= 0 && load_tri_vox(a.tv, a.T, rep, A, B, C)) {
            const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
            uc = sqrtf(closest_d2(p, A, B, C));
            const int dx = ic - si, dy = jc - sj, dz = kc - sk;
            masked = (float)(dx * dx + dy * dy + dz * dz) <= a.mask2;
        }
        // winner record (tracked calls): the coarse source holds a voxel's distance
        // when the voxel is unmasked, starts fresh, or its coarse distance is lower
        bool coarse_wins = true;
        const uint32_t ub = __float_as_uint(uc);
        if (!masked) {
            sdf[lin] = uc - a.beta;
            dist_bits[lin] = ub;
            front[lin] = 0u;
            back[lin] = 0u;
        } else if (a.accumulate == 1) {
            const uint32_t old = dist_bits[lin];
            coarse_wins = ub < old;
            dist_bits[lin] = min(old, ub);
        } else {
            // fresh, or Eq. (1): alpha * f_{t-1} + (1 - alpha) * c_t before this frame's hits
            const float f = a.accumulate == 2 ? a.alpha * __uint_as_float(dist_bits[lin]) + a.one_minus_alpha * uc
                                              : uc;
            dist_bits[lin] = __float_as_uint(f);
            front[lin] = 0u;
            back[lin] = 0u;
        }
        if (win_ray && coarse_wins) {
            win_ray[lin] = 0xFFFFFFFFu;
            win_tri[lin] = -1;
        }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, masked);
    if (tx == 0 && bal) {
        const int shift = ((tz % BZ) * BY + (ty % BY)) * BX;
        const int row = ((tz / BZ) * kBpy + ty / BY) * kBpx;
#pragma unroll
        for (int b = 0; b < kBpx; ++b) {
            const unsigned long long nib = (BX == 32) ? (unsigned long long)bal
                                                      : (unsigned long long)((bal >> (BX * b)) & ((1u << BX) - 1u));
            if (nib) atomicOr(&smask[row + b], nib << shift);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lb = threadIdx.x;
        const int bx = tb.x * kBpx + lb % kBpx, by = tb.y * kBpy + (lb / kBpx) % kBpy,
                  bz = tb.z * (4 / BZ) + lb / (kBpx * kBpy);
        const bool valid = lb < kPer && bx < a.nbx && by < a.nby && bz < a.nbz;
        const unsigned long long m = valid ? smask[lb] : 0ull;
        const int64_t b = ((int64_t)bz * a.nby + by) * a.nbx + bx;
        if (valid) bmask[b] = m;
        const uint32_t act = __ballot_sync(0xffffffffu, m != 0ull);
        uint32_t base = 0;
        if (threadIdx.x == 0 && act) base = atomicAdd(count, (uint32_t)__popc(act));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (m) blist[base + __popc(act & ((1u << threadIdx.x) - 1u))] = tag | (int32_t)b;
    }
}

// Does box [lo, hi] come within `ext` of the box [qlo, qhi] (the voxel centres of a
// brick)?  Every point a ray of the brick can reach satisfies this, so boxes that
// fail it hold no triangle any of the brick's rays can hit.
__device__ __forceinline__ bool box_near(float4 lo, float4 hi, float3 qlo, float3 qhi, float ext2) {
    const float gx = fmaxf(fmaxf(lo.x - qhi.x, qlo.x - hi.x), 0.0f);
    const float gy = fmaxf(fmaxf(lo.y - qhi.y, qlo.y - hi.y), 0.0f);
    const float gz = fmaxf(fmaxf(lo.z - qhi.z, qlo.z - hi.z), 0.0f);
    return __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, gz * gz)) <= ext2;
}

// Warp-cooperative walk of the BVH for the query region: pops up to 32 nodes per
// step from the warp's stack and appends the leaves it reaches to `list`; stops
// when the stack is empty or the list could overflow on the next step.  Returns
// the new list length; `sp` is the stack depth.  A step grows the stack by at most
// the nodes it pops, so once the stack is within kNarrowMargin of its capacity the
// walk pops one node per step (depth first from the top): from there the stack
// grows by at most the tree's depth, which stays below the margin.
__device__ __forceinline__ int walk_and_stage(const BvhNode* __restrict__ nodes, int n_inner, int n_leaves,
                                              float3 qlo, float3 qhi, float ext2, int* stack, int& sp,
                                              int* list, int nc, bool& overflow, uint32_t& box_tests) {
    const int lane = threadIdx.x & 31;
    int guard = 0;
    while (sp > 0 && nc <= kListCap - 64) {
        if (++guard > n_inner + 64) {  // a well-formed tree is exhausted long before
            overflow = true;
            sp = 0;
            break;
        }
        const int take = sp > kStackCapW - kNarrowMargin ? 1 : min(sp, 32);
        box_tests += (uint32_t)(n_leaves > 1 ? 2 * take : take);
        int node = -1;
        if (lane < take) node = stack[sp - 1 - lane];
        sp -= take;
        bool h0 = false, h1 = false;
        int c0 = 0, c1 = 0;
        if (node >= 0 && node < n_inner) {
            const BvhNode* nd = nodes + node;
            const float4 lo0 = __ldg(&nd->lo0), hi0 = __ldg(&nd->hi0);
            const float4 lo1 = __ldg(&nd->lo1), hi1 = __ldg(&nd->hi1);
            c0 = __float_as_int(lo0.w);
            c1 = __float_as_int(hi0.w);
            h0 = box_near(lo0, hi0, qlo, qhi, ext2);
            h1 = n_leaves > 1 && box_near(lo1, hi1, qlo, qhi, ext2);
            if (c0 < 0 && ~c0 >= n_leaves) h0 = false;
            if (c1 < 0 && ~c1 >= n_leaves) h1 = false;
        }
        const int np = (h0 && c0 >= 0) + (h1 && c1 >= 0);
        const int nl = (h0 && c0 < 0) + (h1 && c1 < 0);
        int pp = np, pl = nl;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, pp, off);
            const int v = __shfl_up_sync(0xffffffffu, pl, off);
            if (lane >= off) {
                pp += u;
                pl += v;
            }
        }
        const int tot_p = __shfl_sync(0xffffffffu, pp, 31);
        const int tot_l = __shfl_sync(0xffffffffu, pl, 31);
        int wp = sp + pp - np;
        if (h0 && c0 >= 0) { if (wp < kStackCapW) stack[wp] = c0; ++wp; }
        if (h1 && c1 >= 0) { if (wp < kStackCapW) stack[wp] = c1; ++wp; }
        int wl = nc + pl - nl;
        if (h0 && c0 < 0) list[wl++] = ~c0;
        if (h1 && c1 < 0) list[wl++] = ~c1;
        if (sp + tot_p > kStackCapW) {
            overflow = true;
            sp = kStackCapW;
        } else {
            sp += tot_p;
        }
        nc += tot_l;
        __syncwarp();
    }
    return nc;
}

// Sizes of the per-warp state for RPL rays per lane and group: groups of up to 8 rays
// share one layout; 16-ray groups (9 to 16 rays per voxel) have twice the ray rows.
template <int RPL>
struct RaySlots {
    static constexpr int kRays = RPL <= 8 ? 8 : RPL;  // ray rows of the direction and closest-hit arrays
    static constexpr int kQuads = kRays / 4;
    static constexpr int kRBits = RPL <= 8 ? 3 : 4;   // ray bits of a queued item
    static constexpr int kQueue = 32 + 32 * kRays;    // < 32 left over + one filter round
};

// Resident refine warps per SM for RPL rays per lane and group.
template <int RPL>
constexpr int refine_warps_per_sm() {
    return RPL <= 8 ? kRefineWarpsPerSm : kRefineWarpsPerSm16;
}

// Per-warp shared state of k_refine.
template <int RPL>
struct WarpSmemT {
    int list[kListCap];                          // staged leaves
    int stack[kStackCapW];
    uint32_t queue[RaySlots<RPL>::kQueue];        // (list index << (5 + rbits)) | (slot << rbits) | ray
    int qn;                                      // queued items
    uint32_t okm[32];                            // rays of each slot that drew a direction
    float4 origin[32];                           // voxel centres of the pass's slots (w: linear index)
    float4 dq[3][RaySlots<RPL>::kQuads][32];      // ray directions: [component][ray / 4][slot], rays 4q..4q+3 in x..w
    float4 tsph[32];                             // bounding spheres of the chunk's staged triangles (w: radius^2)
    float4 tpln[32];                             // their planes
    float2 tcon[32];                             // their filter constants (near cone threshold, plane margin)
    uint16_t pairs[160];                         // (slot << 5) | chunk lane: (voxel, triangle) pairs to filter
    unsigned long long key[RaySlots<RPL>::kRays][32];  // closest hit: (t bits << 32) | (id << 1) | front
    unsigned long long work[4];                  // node, reach, filter-pair and exact-test counts (lane 0 writes)
    uint32_t near_edge;                          // exact-test hits within 1e-6 of an edge (lane 0 writes)
};

enum { kWorkNodes = 0, kWorkReach = 1, kWorkPairs = 2, kWorkExact = 3 };

// Work counts of the warp (counting kernels only), kept in its shared state by lane 0
// and added to the caller's counters once per warp (work_flush).
template <int RPL>
__device__ __forceinline__ void work_reset(WarpSmemT<RPL>& w) {
    if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < 4; ++i) w.work[i] = 0ull;
        w.near_edge = 0u;
    }
    __syncwarp();
}



template <int RPL>
__device__ __forceinline__ void work_flush(WarpSmemT<RPL>& w, rtsdf_counters* counters) {
    __syncwarp();
    if (counters && (threadIdx.x & 31) == 0) {
        if (w.work[kWorkNodes]) atomicAdd(reinterpret_cast<unsigned long long*>(&counters->node_tests), w.work[kWorkNodes]);
        if (w.work[kWorkReach]) atomicAdd(reinterpret_cast<unsigned long long*>(&counters->reach_tests), w.work[kWorkReach]);
        if (w.work[kWorkPairs]) atomicAdd(reinterpret_cast<unsigned long long*>(&counters->filter_pairs), w.work[kWorkPairs]);
        if (w.work[kWorkExact]) atomicAdd(reinterpret_cast<unsigned long long*>(&counters->exact_tests), w.work[kWorkExact]);
        if (w.near_edge) atomicAdd(&counters->near_edge_hits, w.near_edge);
    }
}

// Component comp of ray r's direction at a slot (one scalar shared-memory load).
template <int RPL>
__device__ __forceinline__ float dq_comp(const WarpSmemT<RPL>& w, int comp, int r, int slot) {
    return reinterpret_cast<const float*>(&w.dq[comp][r >> 2][slot])[r & 3];
}

// Exact Moller-Trumbore test of one queued (voxel, ray, triangle) item; the
// closest hit per ray (ties to the lower id) is kept with a 64-bit atomicMin.
template <int RPL, bool kCount>
__device__ __forceinline__ bool run_item(WarpSmemT<RPL>& w, const BvhLeaf* __restrict__ leaves, uint32_t item,
                                         float tmax) {
    constexpr int kB = RaySlots<RPL>::kRBits;
    const int c = (int)(item >> (5 + kB)), slot = (int)((item >> kB) & 31u), r = (int)(item & ((1u << kB) - 1u));
    const float4 of = w.origin[slot];
    const float3 o = make_float3(of.x, of.y, of.z),
                 d = make_float3(dq_comp(w, 0, r, slot), dq_comp(w, 1, r, slot), dq_comp(w, 2, r, slot));
    const BvhLeaf* L = leaves + w.list[c];
    const float4 v0 = __ldg(&L->v0), e1f = __ldg(&L->e1), e2f = __ldg(&L->e2);
    const float3 A = make_float3(v0.x, v0.y, v0.z);
    const float3 e1 = make_float3(e1f.x, e1f.y, e1f.z), e2 = make_float3(e2f.x, e2f.y, e2f.z);
    float t, margin;
    bool front;
    const bool hit = ray_tri_flat(o, d, A, e1, e2, tmax, t, front, margin);
    if (hit) {
        const uint32_t id = (uint32_t)__float_as_int(v0.w);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)((id << 1) | (front ? 1u : 0u));
        atomicMin(&w.key[r][slot], key);
    }
    return hit && margin < 1e-6f;
}

// Work counts of one brick, the same in every lane (added to the warp's shared totals
// once per brick, at the end of refine_brick).
struct BrickWork {
    uint32_t pairs = 0, exact = 0, near = 0;
};

// Lane 0 adds n to the warp's shared count i (outside the hot loops: once per BVH walk).
template <int RPL>
__device__ __forceinline__ void work_add(WarpSmemT<RPL>& w, int i, uint32_t n) {
    if ((threadIdx.x & 31) == 0) w.work[i] += n;
}

// Exact tests of the items of the first n lanes (items[lane]); with kCount, counted.
template <int RPL, bool kCount>
__device__ __forceinline__ void run_items(WarpSmemT<RPL>& w, const BvhLeaf* __restrict__ leaves, const uint32_t* items,
                                          int n, float tmax, BrickWork& bw) {
    const int lane = threadIdx.x & 31;
    if (kCount) {
        const bool near = lane < n && run_item<RPL, true>(w, leaves, items[lane], tmax);
        bw.exact += (uint32_t)n;
        bw.near += (uint32_t)__popc(__ballot_sync(0xffffffffu, near));
    } else if (lane < n) {
        run_item<RPL, false>(w, leaves, items[lane], tmax);
    }
}

// Slab test of a ray against box [lo, hi]: iv the inverse direction components, no =
// -o * iv, so the box's planes are crossed at t = lo * iv + no.  tn receives the entry
// parameter (at least -1e-3); the box counts as hit when the entry is at most the exit
// and at most lim, each with 1e-3 (voxel lengths; d is a unit vector) to spare.
__device__ __forceinline__ bool ray_box(float4 lo, float4 hi, float3 iv, float3 no, float lim, float& tn) {
    const float ax = __fmaf_rn(lo.x, iv.x, no.x), bx = __fmaf_rn(hi.x, iv.x, no.x);
    const float ay = __fmaf_rn(lo.y, iv.y, no.y), by = __fmaf_rn(hi.y, iv.y, no.y);
    const float az = __fmaf_rn(lo.z, iv.z, no.z), bz = __fmaf_rn(hi.z, iv.z, no.z);
    tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), -1e-3f));
    const float tf = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
    return tn <= tf + 1e-3f && tn <= lim;
}

constexpr int kRayStack = 64;  // per-lane traversal stack: a radix tree over unique 64-bit keys is at most 64 deep

// Closest hit of one ray (origin o, unit direction d, length tmax) over the whole
// BVH, by a depth-first walk of the lane's own: both child boxes of a node get the
// slab test, the nearer child is entered and the other pushed, and each leaf gets
// the exact test of run_item (the same function, operands and key), so `best` is the
// lowest key over all triangles, the one the staged path finds.  The boxes carry
// the builder's padding (at least 1/64 voxel), far above the FP32 rounding of the
// slab parameters (about 1e-7 of the coordinates) and of any accepted hit point, so
// no box holding a hit is skipped; directions are kept at least 1e-12 from zero in
// each component, which keeps every parameter finite and moves the ray by far less
// than that padding.  Without kCount a box entered beyond the closest hit so far is
// skipped (a hit inside it lies at or beyond its entry, so its key is not lower);
// with kCount every box within the ray's length is opened, so that, as in the
// staged path, the exact test sees every triangle the ray can hit and the near-edge
// count covers every hit.  Returns false if the stack or the step guard would
// overflow, which a tree from the builder never does; the caller counts the brick
// like a walk that overflowed.
template <bool kCount>
__device__ __forceinline__ bool ray_closest(const BvhNode* __restrict__ nodes, const BvhLeaf* __restrict__ leaves,
                                            int n_leaves, int n_inner, float3 o, float3 d, float tmax,
                                            unsigned long long& best, uint32_t& box_tests, uint32_t& exact,
                                            uint32_t& near) {
    int stk[kRayStack];
    float stn[kRayStack];
    const float tiny = 1e-12f;
    const float3 iv = make_float3(__frcp_rn(fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                                  __frcp_rn(fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                                  __frcp_rn(fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float3 no = make_float3(-o.x * iv.x, -o.y * iv.y, -o.z * iv.z);
    best = ~0ull;
    if (n_leaves <= 0) return true;
    float lim = tmax * 1.000001f + 1e-3f;  // boxes entered beyond lim hold no lower key
    int sp = 0, node = 0, guard = 0;
    auto leaf = [&](int j) {
        const BvhLeaf* L = leaves + j;
        const float4 v0 = __ldg(&L->v0), e1f = __ldg(&L->e1), e2f = __ldg(&L->e2);
        float t, margin;
        bool front;
        const bool hit = ray_tri_flat(o, d, make_float3(v0.x, v0.y, v0.z), make_float3(e1f.x, e1f.y, e1f.z),
                                      make_float3(e2f.x, e2f.y, e2f.z), tmax, t, front, margin);
        if (kCount) {
            ++exact;
            near += (hit && margin < 1e-6f) ? 1u : 0u;
        }
        if (hit) {
            const uint32_t id = (uint32_t)__float_as_int(v0.w);
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)((id << 1) | (front ? 1u : 0u));
            if (key < best) {
                best = key;
                if (!kCount) lim = t * 1.000001f + 1e-3f;
            }
        }
    };
    while (true) {
        if (++guard > n_inner + 1) return false;  // a tree's walk enters each inner node once
        const BvhNode* nd = nodes + node;
        const float4 lo0 = __ldg(&nd->lo0), hi0 = __ldg(&nd->hi0), lo1 = __ldg(&nd->lo1), hi1 = __ldg(&nd->hi1);
        const int c0 = __float_as_int(lo0.w), c1 = __float_as_int(hi0.w);
        float t0 = 0.f, t1 = 0.f;
        bool h0 = ray_box(lo0, hi0, iv, no, lim, t0) && (c0 >= 0 ? c0 < n_inner : ~c0 < n_leaves);
        bool h1 = n_leaves > 1 && ray_box(lo1, hi1, iv, no, lim, t1) && (c1 >= 0 ? c1 < n_inner : ~c1 < n_leaves);
        if (kCount) box_tests += n_leaves > 1 ? 2u : 1u;
        if (h0 && c0 < 0) {
            leaf(~c0);
            h0 = false;
        }
        if (h1 && c1 < 0) {
            leaf(~c1);
            h1 = false;
        }
        if (h0 && h1) {
            if (sp >= kRayStack) return false;
            const bool n0 = t0 <= t1;
            stk[sp] = n0 ? c1 : c0;
            stn[sp] = n0 ? t1 : t0;
            ++sp;
            node = n0 ? c0 : c1;
        } else if (h0 || h1) {
            node = h0 ? c0 : c1;
        } else {
            // pop the next pushed node still entered within lim
            do {
                if (sp == 0) return true;
                --sp;
            } while (stn[sp] > lim);
            node = stk[sp];
        }
    }
}

// Which rays of one (voxel slot v, staged triangle) pair can hit the triangle.  Two
// necessary conditions, each a dot product of the ray direction d with a per-pair
// vector against a per-pair threshold:
//  - the line of the ray passes within rho of the triangle's bounding sphere centre
//    c, with the centre at most rho behind the origin: tc = (c - o).d >= thr, where
//    off the rho-sphere by more than rho*sqrt(2) thr = sqrt(|c - o|^2 - rho^2) is the
//    exact cone, and nearer thr = -rho (every point of the sphere at t >= 0 has
//    tc >= t - rho >= -rho);
//  - the ray crosses the triangle's plane at t_p = sd / dn in [0, tmax] (sd the
//    signed distance of the plane from the origin, dn = n.d).  That holds exactly
//    when sd*dn >= sd^2 / tmax (the parabola f(sd) = sd*dn - sd^2/tmax is
//    non-negative between its roots 0 and tmax*dn), so with m = sd*n the test is
//    m.d >= sd^2/tmax - M.  The margin M = 1.5 eps + eps^2/tmax covers every sd in
//    [-eps, tmax*dn + eps], the plane crossing widened by eps in sd (where f >=
//    -(eps |dn| + eps^2/tmax)), with eps/2 to spare for rounding.
// Each threshold is folded into the first FMA of its dot product, so a ray passes
// when both results are non-negative: the OR of their bit patterns has a clear sign
// bit, and a funnel shift appends that bit to the pair's mask.  All margins exceed
// the FP32 rounding of both sides (values of at most a few tens of voxels; 1e-4
// absolute and 1e-6 relative in the cone, eps >= 2e-3 in the plane), so no triangle
// the exact test accepts is dropped.
template <int RPL>
__device__ __forceinline__ uint32_t filter_pair(const WarpSmemT<RPL>& w, int v, int j, float tmax, float inv_tmax) {
    constexpr int kQ = (RPL + 3) / 4;
    const float4 o = w.origin[v];
    const float4 sph = w.tsph[j], pl = w.tpln[j];  // sph.w: rho^2
    const float2 tk = w.tcon[j];
    const float dcx = sph.x - o.x, dcy = sph.y - o.y, dcz = sph.z - o.z;
    const float dd = __fmaf_rn(dcx, dcx, __fmaf_rn(dcy, dcy, dcz * dcz));
    // v * rsqrt(v) is within a few ulp of sqrt(v) (a few 1e-7 relative), well inside the
    // 1e-6 relative and 1e-4 absolute margins, so the threshold stays below the exact one;
    // v2 > rho^2 (the origin farther than about rho sqrt(2)) keeps v2 well above 0
    const float v2 = dd - sph.w;
    const float thr = v2 > sph.w ? (v2 * rsqrtf(v2)) * 0.999999f - 1e-4f : tk.x;
    const float sd = pl.w - __fmaf_rn(pl.x, o.x, __fmaf_rn(pl.y, o.y, pl.z * o.z));
    const float bq = __fmaf_rn(sd * inv_tmax, sd, -tk.y);
    const float2 cx2 = make_float2(dcx, dcx), cy2 = make_float2(dcy, dcy), cz2 = make_float2(dcz, dcz);
    const float2 mx2 = make_float2(sd * pl.x, sd * pl.x), my2 = make_float2(sd * pl.y, sd * pl.y),
                 mz2 = make_float2(sd * pl.z, sd * pl.z);
    const float2 nthr2 = make_float2(-thr, -thr), nbq2 = make_float2(-bq, -bq);
    uint32_t fail = 0;  // bit r set: ray r fails one of the tests
#pragma unroll
    for (int q = kQ - 1; q >= 0; --q) {
        const float4 qx = w.dq[0][q][v], qy = w.dq[1][q][v], qz = w.dq[2][q][v];
        const float2 xs[2] = {make_float2(qx.x, qx.y), make_float2(qx.z, qx.w)};
        const float2 ys[2] = {make_float2(qy.x, qy.y), make_float2(qy.z, qy.w)};
        const float2 zs[2] = {make_float2(qz.x, qz.y), make_float2(qz.z, qz.w)};
#pragma unroll
        for (int hq = (RPL >= 4 ? 1 : 0); hq >= 0; --hq) {
            const float2 tc = __ffma2_rn(cx2, xs[hq], __ffma2_rn(cy2, ys[hq], __ffma2_rn(cz2, zs[hq], nthr2)));
            const float2 pp = __ffma2_rn(mx2, xs[hq], __ffma2_rn(my2, ys[hq], __ffma2_rn(mz2, zs[hq], nbq2)));
            // rays are appended from the highest index down, so ray r ends at bit r
            fail = __funnelshift_l(__float_as_uint(tc.y) | __float_as_uint(pp.y), fail, 1);
            fail = __funnelshift_l(__float_as_uint(tc.x) | __float_as_uint(pp.x), fail, 1);
        }
    }
    return ~fail & w.okm[v];
}

// Exact tests of full batches of 32 queued items.
template <int RPL, bool kCount>
__device__ __forceinline__ void run_full_batches(WarpSmemT<RPL>& w, const BvhLeaf* __restrict__ leaves, float tmax,
                                                 BrickWork& bw) {
    const int lane = threadIdx.x & 31;
    int qn = w.qn;
    if (qn >= 32) {
        while (qn >= 32) {
            run_items<RPL, kCount>(w, leaves, w.queue + (qn - 32), 32, tmax, bw);
            qn -= 32;
        }
        __syncwarp();
        if (lane == 0) w.qn = qn;
    }
    __syncwarp();
}

// Filters one (voxel slot, chunk triangle) pair per lane (lanes >= n idle) and queues
// the surviving (voxel, ray, triangle) items.
template <int RPL, bool kCount>
__device__ __forceinline__ void filter_and_queue(WarpSmemT<RPL>& w, int n, int base, int cb, float tmax,
                                                 float inv_tmax, BrickWork& bw) {
    const int lane = threadIdx.x & 31;
    if (kCount) bw.pairs += (uint32_t)n;
    if (lane < n) {
        const uint32_t p = w.pairs[base + lane];
        const int v = (int)(p >> 5), j = (int)(p & 31u);
        uint32_t pm = filter_pair<RPL>(w, v, j, tmax, inv_tmax);
        if (pm) {
            int pos = atomicAdd(&w.qn, __popc(pm));
            while (pm) {
                const int r = __ffs(pm) - 1;
                pm &= pm - 1u;
                w.queue[pos++] = ((uint32_t)(cb + j) << (5 + RaySlots<RPL>::kRBits)) |
                                 ((uint32_t)v << RaySlots<RPL>::kRBits) | (uint32_t)r;
            }
        }
    }
    __syncwarp();
}

// (Voxel, triangle group) combinations of a staged chunk that can produce a hit.  The
// chunk's four groups of 8 triangles (lanes 8g .. 8g + 7, lane j holding triangle j's
// bounding sphere, valid when `have`) each get a sphere around the box of their
// triangles' spheres, grown by a margin above FP32 rounding; every voxel of the pass
// (lane v < nv) tests its rays against the four like a triangle's sphere in
// filter_pair: a group out of the voxel's reach, or whose sphere every ray line
// misses, holds no triangle any of the voxel's rays can hit.  Returns the voxels with
// some group left (bit v) and sets, in lane v, the 4-bit mask of its groups (bit g);
// the voxel's pairs are formed with those groups' triangles only.  On coarse grids,
// where a brick stages thousands of triangles within reach of its voxels, most
// combinations fail and their pairs are never formed.
template <int RPL>
__device__ __forceinline__ uint32_t chunk_voxels(const WarpSmemT<RPL>& w, float4 sph, bool have, int nv,
                                                  float tmax, uint32_t& groups) {
    constexpr int kQ = (RPL + 3) / 4;
    const int lane = threadIdx.x & 31;
    const float inf = __int_as_float(0x7f800000);
    float lx = have ? sph.x - sph.w : inf, ly = have ? sph.y - sph.w : inf, lz = have ? sph.z - sph.w : inf;
    float hx = have ? sph.x + sph.w : -inf, hy = have ? sph.y + sph.w : -inf, hz = have ? sph.z + sph.w : -inf;
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {  // within each group of 8 lanes
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, off));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, off));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, off));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, off));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, off));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, off));
    }
    const bool gvalid = lx <= hx;  // the group holds a staged triangle
    const float gx = 0.5f * (lx + hx), gy = 0.5f * (ly + hy), gz = 0.5f * (lz + hz);
    const float ex = hx - lx, ey = hy - ly, ez = hz - lz;
    const float grho =
        gvalid ? 0.5f * sqrtf(__fmaf_rn(ex, ex, __fmaf_rn(ey, ey, ez * ez))) * 1.00001f + 1e-3f : 0.0f;
    const float4 o = w.origin[lane];
    const bool mine = lane < nv;
    uint32_t m = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float cx = __shfl_sync(0xffffffffu, gx, 8 * g), cy = __shfl_sync(0xffffffffu, gy, 8 * g),
                    cz = __shfl_sync(0xffffffffu, gz, 8 * g), rho = __shfl_sync(0xffffffffu, grho, 8 * g);
        const bool valid = __shfl_sync(0xffffffffu, gvalid, 8 * g);
        const float dcx = cx - o.x, dcy = cy - o.y, dcz = cz - o.z;
        const float dd = __fmaf_rn(dcx, dcx, __fmaf_rn(dcy, dcy, dcz * dcz));
        const float reach = rho + tmax * 1.00001f + 1e-3f;
        bool pass = mine && valid && dd <= reach * reach;
        if (pass) {
            const float rho2 = rho * rho;
            const float v2 = dd - rho2;
            const float thr = v2 > rho2 ? (v2 * rsqrtf(v2)) * 0.999999f - 1e-4f : -rho * 1.000001f - 1e-4f;
            const float2 cx2 = make_float2(dcx, dcx), cy2 = make_float2(dcy, dcy), cz2 = make_float2(dcz, dcz);
            const float2 nthr2 = make_float2(-thr, -thr);
            uint32_t any = 0;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const float4 qx = w.dq[0][q][lane], qy = w.dq[1][q][lane], qz = w.dq[2][q][lane];
                const float2 t0 = __ffma2_rn(cx2, make_float2(qx.x, qx.y),
                                             __ffma2_rn(cy2, make_float2(qy.x, qy.y),
                                                        __ffma2_rn(cz2, make_float2(qz.x, qz.y), nthr2)));
                const float2 t1 = __ffma2_rn(cx2, make_float2(qx.z, qx.w),
                                             __ffma2_rn(cy2, make_float2(qy.z, qy.w),
                                                        __ffma2_rn(cz2, make_float2(qz.z, qz.w), nthr2)));
                any |= ~(__float_as_uint(t0.x) & __float_as_uint(t0.y) & __float_as_uint(t1.x) &
                         __float_as_uint(t1.y));
            }
            pass = (any >> 31) != 0u;
        }
        m |= pass ? 1u << g : 0u;
    }
    groups = m;
    return __ballot_sync(0xffffffffu, m != 0u);
}

// Position of the n-th set bit (from 0) of m, n < popc(m): a binary search on
// population counts, the same few steps in every lane.
__device__ __forceinline__ int nth_set_bit(unsigned long long m, int n) {
    int pos = 0;
    uint32_t x = (uint32_t)m;
    const int lo = __popc(x);
    if (n >= lo) {
        n -= lo;
        x = (uint32_t)(m >> 32);
        pos = 32;
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(x & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Lists the (slot, ray) items of the warp's rays in its item queue, which holds
// 32 * RPL of them: bit r of m in lane l gives item (l << 5) | r, lanes in order.
// Returns the number of items; called by the whole warp.
template <int RPL>
__device__ __forceinline__ int list_rays(WarpSmemT<RPL>& w, uint32_t m) {
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - cnt;
    while (m) {
        const int r = __ffs(m) - 1;
        m &= m - 1u;
        w.queue[pos++] = ((uint32_t)lane << 5) | (uint32_t)r;
    }
    __syncwarp();
    return total;
}

// Rays of the group whose first draw failed (both candidate pairs of attempt 0
// rejected, about 4.6% of rays; bit r of `need` in the lane owning the slot) continue
// from attempt 1, one ray per lane: the warp lists its (slot, ray) items in the item
// queue, which is unused at this point, so a retry costs one round of draws for up to
// 32 rays instead of a loop per ray row that nearly every warp would enter.  Each
// success writes the ray's direction into the slot's row and sets its bit in okm;
// rays that fail all 32 attempts are counted in n_fail.  Called by the whole warp.
template <int RPL>
__device__ __forceinline__ void redraw(WarpSmemT<RPL>& w, uint32_t need, const RefineArgs& a, int r0,
                                       uint32_t& n_fail) {
    const int lane = threadIdx.x & 31;
    const int total = list_rays<RPL>(w, need);
    for (int b = 0; b < total; b += 32) {
        if (b + lane < total) {
            const uint32_t it = w.queue[b + lane];
            const int slot = (int)(it >> 5), r = (int)(it & 31u);
            const uint32_t vox = (uint32_t)__float_as_int(w.origin[slot].w);
            float3 d;
            if (sphere_dir(vox, a.frame * (uint32_t)a.R + (uint32_t)(r0 + r), a.scene, a.k0, a.k1, d, 1u)) {
                float* row = reinterpret_cast<float*>(&w.dq[0][r >> 2][slot]);
                row[r & 3] = d.x;
                reinterpret_cast<float*>(&w.dq[1][r >> 2][slot])[r & 3] = d.y;
                reinterpret_cast<float*>(&w.dq[2][r >> 2][slot])[r & 3] = d.z;
                atomicOr(&w.okm[slot], 1u << r);
            } else {
                ++n_fail;
            }
        }
    }
    __syncwarp();
}

// One warp refines one brick (bx, by, bz) whose masked voxels are the set bits of
// m; lane l owns voxel slot (pass*32 + l) and draws up to 8 rays of it per group.
// The brick's staged triangles are taken 32 at a time (one per lane): every
// (voxel slot, triangle) pair within reach of the triangle's bounding sphere grown
// by the ray length is compacted into a pair list, four voxels per step, and the
// pairs are filtered 32 at a time, one per lane, against all rays of the voxel (the
// line of each ray must pass the sphere, and the ray must cross the triangle's
// plane within its length).  So the filter does no work for pairs out of reach
// and none for empty slots of a partly filled pass.  Surviving (voxel, ray,
// triangle) items are queued in shared memory and run through the exact
// ray/triangle test 32 at a time, so the expensive test does not diverge.  The
// filters are conservative (their margins exceed FP32 rounding of the exact test),
// so they never drop a triangle the exact test accepts; they may use fused
// multiply-adds because they decide nothing the oracle decides.
// RPL: rays per lane and group (2, 4 or 8); calls with R <= RPL rays per voxel run
// one group, so small ray counts do not pay for eight.
// With kCull and a.per_ray, a brick whose walk overflows its list (more than
// kListCap - 64 triangles within reach of its rays) is not refined here: the call
// returns true and the caller lists the brick for a second launch with kRays, in
// which every ray of the brick walks the BVH on its own (ray_closest) and nothing
// is staged.  The two paths live in separate kernels so that the staged one keeps
// its registers.
template <int BX, int BY, int BZ, bool kTrack, int RPL = kRaysPerLane, bool kCount = false, bool kCull = false,
          bool kRays = false>
__device__ __forceinline__ bool refine_brick(const RefineArgs& a, const BvhNode* __restrict__ nodes,
                                             const BvhLeaf* __restrict__ leaves, int n_leaves, int n_inner,
                                             const int32_t* __restrict__ nearest,
                                             const int32_t* __restrict__ rep_tri, unsigned long long m, int bx,
                                             int by, int bz, uint32_t* __restrict__ dist_bits,
                                             uint32_t* __restrict__ front, uint32_t* __restrict__ back,
                                             float* __restrict__ sdf, uint32_t* __restrict__ win_ray,
                                             int32_t* __restrict__ win_tri, WarpSmemT<RPL>& w, uint32_t& n_hit,
                                             uint32_t& n_fail, uint32_t& n_ovf) {
    const int lane = threadIdx.x & 31;
    const float ext = a.tmax * 1.00001f + 1e-3f;
    const float inv_tmax = 1.0f / a.tmax;
    const int nm = __popcll(m);
    // every ray of the brick stays inside its voxel centres' box grown by the ray length
    const float3 qlo = make_float3((float)(bx * BX) + 0.5f, (float)(by * BY) + 0.5f, (float)(bz * BZ) + 0.5f);
    const float3 qhi = make_float3((float)(bx * BX + BX - 1) + 0.5f, (float)(by * BY + BY - 1) + 0.5f,
                                   (float)(bz * BZ + BZ - 1) + 0.5f);
    bool overflow = false;
    // walk once for the whole brick; the list is reused by every pass and ray
    // group unless it overflowed, in which case each pass walks again in rounds
    int sp0 = 0;
    if (!kRays && n_leaves > 0) {
        if (lane == 0) w.stack[0] = 0;
        sp0 = 1;
    }
    __syncwarp();
    BrickWork bw;
    uint32_t box_tests = 0;
    const int nc_all = kRays ? 0
                             : walk_and_stage(nodes, n_inner, n_leaves, qlo, qhi, ext * ext, w.stack, sp0, w.list, 0,
                                              overflow, box_tests);
    if (kCount) work_add(w, kWorkNodes, box_tests);
    const bool complete = !kRays && sp0 == 0;
    if (kCull && !kRays && a.per_ray && !complete) return true;  // for the per-ray launch
    for (int pass = 0; pass * 32 < nm; ++pass) {
        const int slot = pass * 32 + lane;
        const bool mine = slot < nm;
        int lin = 0;
        int64_t clin = 0;  // coarse voxel of the slot (its flooded seed)
        float3 o = make_float3(0.f, 0.f, 0.f);
        if (mine) {
            const int bit = nth_set_bit(m, slot);
            const int i = bx * BX + bit % BX, j = by * BY + (bit / BX) % BY, k = bz * BZ + bit / (BX * BY);
            lin = (int)(((int64_t)k * a.g.ny + j) * a.g.nx + i);
            int ic, jc, kc;
            clin = coarse_index(a, i, j, k, ic, jc, kc);
            o = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
        }
        w.origin[lane] = make_float4(o.x, o.y, o.z, __int_as_float(lin));  // w: the voxel's linear index
        const int nv = min(32, nm - pass * 32);
        uint32_t vbest = 0xffffffffu, vfront = 0, vback = 0;
        // tracked: this call's winning ray, ordered by (t, triangle id), first ray on ties
        unsigned long long wkey = ~0ull;
        uint32_t wray = 0xFFFFFFFFu;
        for (int r0 = 0; r0 < a.R; r0 += RPL) {
            float3 dir[RPL];
            uint32_t okm = 0, need = 0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int ray = r0 + r;
                dir[r] = make_float3(0.f, 0.f, 1.f);
                if (mine && ray < a.R) {
                    if (sphere_dir_first((uint32_t)lin, a.frame * (uint32_t)a.R + (uint32_t)ray, a.scene, a.k0,
                                         a.k1, dir[r]))
                        okm |= 1u << r;
                    else
                        need |= 1u << r;
                }
                w.key[r][lane] = ~0ull;
            }
#pragma unroll
            for (int q = 0; q < (RPL + 3) / 4; ++q) {
                float c[3][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = 4 * q + e;
                    c[0][e] = r < RPL ? dir[r < RPL ? r : 0].x : 0.f;
                    c[1][e] = r < RPL ? dir[r < RPL ? r : 0].y : 0.f;
                    c[2][e] = r < RPL ? dir[r < RPL ? r : 0].z : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) w.dq[k][q][lane] = make_float4(c[k][0], c[k][1], c[k][2], c[k][3]);
            }
            w.okm[lane] = okm;
            if (__any_sync(0xffffffffu, need != 0u)) redraw<RPL>(w, need, a, r0, n_fail);
            __syncwarp();
            bool staged = !kRays;
            if (kRays) {
                // the pass's rays, 32 at a time over the lanes whatever their voxels
                bool done = true;
                uint32_t nb = 0, ne = 0, nn = 0;
                const int total = list_rays<RPL>(w, w.okm[lane]);
                for (int b = 0; b < total; b += 32) {
                    if (b + lane < total) {
                        const uint32_t it = w.queue[b + lane];
                        const int sl = (int)(it >> 5), r = (int)(it & 31u);
                        const float4 of = w.origin[sl];
                        const float3 dd = make_float3(dq_comp(w, 0, r, sl), dq_comp(w, 1, r, sl),
                                                      dq_comp(w, 2, r, sl));
                        unsigned long long key;
                        done = ray_closest<kCount>(nodes, leaves, n_leaves, n_inner, make_float3(of.x, of.y, of.z),
                                                   dd, a.tmax, key, nb, ne, nn) && done;
                        w.key[r][sl] = key;
                    }
                }
                if (kCount) {
                    work_add(w, kWorkNodes, __reduce_add_sync(0xffffffffu, nb));
                    bw.exact += __reduce_add_sync(0xffffffffu, ne);
                    bw.near += __reduce_add_sync(0xffffffffu, nn);
                }
                // a malformed tree (never built): counted like a walk that overflowed
                if (!done) overflow = true;
                __syncwarp();
            }
            int sp = 0;
            if (staged && !complete && n_leaves > 0) {
                if (lane == 0) w.stack[0] = 0;
                sp = 1;
            }
            __syncwarp();
            bool first = staged;
            while (first || sp > 0) {
                first = false;
                box_tests = 0;
                const int nc = complete ? nc_all
                                        : walk_and_stage(nodes, n_inner, n_leaves, qlo, qhi, ext * ext, w.stack,
                                                         sp, w.list, 0, overflow, box_tests);
                // every (voxel, staged triangle) pair of the pass meets the reach test
                if (kCount) {
                    work_add(w, kWorkNodes, box_tests);
                    work_add(w, kWorkReach, (uint32_t)(nv * nc));
                }
                if (lane == 0) w.qn = 0;
                __syncwarp();
                for (int cb = 0; cb < nc; cb += 32) {
                    // lane j holds staged triangle cb + j; pairs (voxel slot, j) that pass the
                    // bounding-sphere reach test are compacted and filtered 32 at a time
                    const int c = cb + lane;
                    float4 sph = make_float4(0.f, 0.f, 0.f, 0.f);
                    float reach2 = -1.0f;
                    if (c < nc) {
                        const BvhLeaf* L = leaves + w.list[c];
                        sph = __ldg(&L->sph);
                        const float4 pl = __ldg(&L->pln);
                        w.tsph[lane] = make_float4(sph.x, sph.y, sph.z, sph.w * sph.w);
                        w.tpln[lane] = pl;
                        // the filter's per-triangle constants: the near cone threshold
                        // -rho (widened) and the plane margin 1.5 eps + eps^2 / tmax
                        const float eps = 2e-3f + 2e-6f * fabsf(pl.w);
                        w.tcon[lane] = make_float2(-sph.w * 1.000001f - 1e-4f,
                                                   __fmaf_rn(eps * eps, inv_tmax, 1.5f * eps));
                        const float reach = sph.w + a.tmax;
                        reach2 = reach * reach;
                    }
                    __syncwarp();
                    // the chunk's voxels: with kCull, on bricks that stage many triangles, those
                    // with a ray that can reach any triangle of the chunk; else all of them
                    uint32_t groups = 0xFu;  // lane v: the triangle groups voxel v is paired with
                    const uint32_t vsel = kCull && nc >= kCullMinStaged
                                              ? chunk_voxels<RPL>(w, sph, c < nc, nv, a.tmax, groups)
                                              : 0xffffffffu;
                    int np = 0;
                    const uint32_t lt = (1u << lane) - 1u;
                    for (int v0 = 0; v0 < nv; v0 += 4) {
                        if (((vsel >> v0) & 0xFu) == 0u) continue;  // four culled voxels (warp-uniform)
                        bool ok[4];
                        uint32_t b[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int v = v0 + e;
                            const float4 ov = w.origin[v & 31];
                            const float dcx = sph.x - ov.x, dcy = sph.y - ov.y, dcz = sph.z - ov.z;
                            const float dd = __fmaf_rn(dcx, dcx, __fmaf_rn(dcy, dcy, dcz * dcz));
                            const uint32_t gv = kCull ? __shfl_sync(0xffffffffu, groups, v & 31) : 0xFu;
                            ok[e] = v < nv && ((vsel >> (v & 31)) & 1u) && ((gv >> (lane >> 3)) & 1u) &&
                                    dd <= reach2;
                            b[e] = __ballot_sync(0xffffffffu, ok[e]);
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (ok[e]) w.pairs[np + __popc(b[e] & lt)] = (uint16_t)(((v0 + e) << 5) | lane);
                            np += __popc(b[e]);
                        }
                        while (np >= 32) {
                            __syncwarp();
                            np -= 32;
                            filter_and_queue<RPL, kCount>(w, 32, np, cb, a.tmax, inv_tmax, bw);
                            run_full_batches<RPL, kCount>(w, leaves, a.tmax, bw);
                        }
                    }
                    __syncwarp();
                    if (np > 0) {
                        filter_and_queue<RPL, kCount>(w, np, 0, cb, a.tmax, inv_tmax, bw);
                        run_full_batches<RPL, kCount>(w, leaves, a.tmax, bw);
                    }
                }
                {
                    const int qn = w.qn;
                    run_items<RPL, kCount>(w, leaves, w.queue, qn, a.tmax, bw);
                    __syncwarp();
                }
                __syncwarp();
                __syncwarp();
            }
            // closest hits of this lane's rays
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const unsigned long long key = w.key[r][lane];
                if (key != ~0ull) {
                    vbest = min(vbest, (uint32_t)(key >> 32));
                    if (key & 1ull) ++vfront; else ++vback;
                    ++n_hit;
                    if (kTrack && (key >> 1) < wkey) {
                        wkey = key >> 1;
                        wray = a.frame * (uint32_t)a.R + (uint32_t)(r0 + r);
                    }
                }
            }
            __syncwarp();
        }
        if (mine) {
            const uint32_t old = dist_bits[lin];
            const uint32_t d = min(old, vbest);
            if (kTrack && vbest < old) {
                win_ray[lin] = wray;
                win_tri[lin] = (int32_t)(wkey & 0x7FFFFFFFull);
            }
            const uint32_t fr = front[lin] + vfront, bk = back[lin] + vback;
            dist_bits[lin] = d;
            front[lin] = fr;
            back[lin] = bk;
            bool neg = bk > fr;
            if (fr == bk && a.fallback) {
                const int32_t s = nearest[clin];
                const int64_t sl2 =
                    ((int64_t)((s >> 20) & 1023) * a.cny + ((s >> 10) & 1023)) * a.cnx + (s & 1023);
                float3 A = make_float3(0.f, 0.f, 0.f), B = A, C = A;
                load_tri_vox(a.tv, a.T, rep_tri[sl2], A, B, C);
                const float3 n = cross3(sub3(B, A), sub3(C, A));
                neg = dot3(sub3(o, A), n) < 0.0f;
            }
            const float df = __uint_as_float(d);
            sdf[lin] = neg ? -df : df;
        }
        __syncwarp();
    }
    if (kCount && lane == 0) {
        w.work[kWorkPairs] += bw.pairs;
        w.work[kWorkExact] += bw.exact;
        w.near_edge += bw.near;
    }
    n_ovf += __any_sync(0xffffffffu, overflow) ? 1u : 0u;
    return false;
}

}  // namespace rtsdf
