// Coarse field, ray mask and ray-sampled refinement (Sec. 2.1-2.3).
//
//  k_resolve: one thread per voxel, blocks of 32x4x4 voxels = 8 bricks of 4^3.
//             Coarse distance u_c to the representative triangle of the flooded
//             seed (read from the BVH's voxel-space triangle table); unmasked
//             voxels get their final value (u_c - beta); masked voxels initialise
//             their refine state.  Per brick a 64-bit mask of its masked voxels is
//             assembled from warp ballots, and bricks with any masked voxel are
//             appended to a work list.
//  k_refine:  persistent, one warp per 4^3 brick (two independent warps per
//             64-thread CTA).  The warp walks the BVH once for the whole brick with
//             the box every ray of the brick stays inside (voxel centres grown by
//             the ray length) and stages the overlapping triangles in shared
//             memory; each lane owns one masked voxel and draws its rays.  The
//             (voxel, triangle) pairs within reach are compacted and filtered one
//             per lane against the voxel's rays, and the surviving (voxel, ray,
//             triangle) items get the exact test 32 at a time.  The closest hit of
//             each ray (ties to the lower triangle id) lowers the voxel's distance
//             and adds one front/back vote; the lane then writes the accumulated
//             state and the signed value.  Staging runs in rounds when a brick has
//             more candidates than the buffer holds.  On coarse grids (a staged-
//             triangle estimate above a threshold that grows with the ray count)
//             a brick whose walk overflows the list is left to a second launch
//             instead, k_refine<..., kRays>, in which each ray walks the BVH on its
//             own (slab tests, nearer child first, boxes beyond the closest hit so
//             far skipped) and nothing is staged.
#include "refine_core.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

constexpr int kBX = 4, kBY = 4, kBZ = 4;  // brick shape of the single-scene path
constexpr int kRefineThreads = 64;        // two independent warps per CTA

struct RefineWs {
    uint32_t* count;            // [0] active bricks, [1] work counter, [2] walks that overflowed,
                                // [3] bricks left to the per-ray launch, [4] its work counter
    unsigned long long* bmask;  // per brick: bit (lz*16 + ly*4 + lx) set for masked voxels
    int32_t* blist;             // active bricks
    int32_t* dlist;             // bricks left to the per-ray launch
};

static size_t nbricks(const rtsdf_grid& g) {
    return (size_t)((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY) * ((g.nz + kBZ - 1) / kBZ);
}

static size_t refine_ws_layout(const rtsdf_grid& g, char* base, RefineWs* w) {
    const size_t nb = nbricks(g);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes, 256);
        return p;
    };
    char* c = take(64);
    char* m = take(8 * nb);
    char* l = take(4 * nb);
    char* d = take(4 * nb);
    if (w) {
        w->count = reinterpret_cast<uint32_t*>(c);
        w->bmask = reinterpret_cast<unsigned long long*>(m);
        w->blist = reinterpret_cast<int32_t*>(l);
        w->dlist = reinterpret_cast<int32_t*>(d);
    }
    return off;
}

size_t refine_workspace(const rtsdf_grid& g) { return refine_ws_layout(g, nullptr, nullptr); }

// ------------------------------------------------------------------ resolve

// Latency-bound (a chain of dependent loads per voxel: flooded seed, representative
// triangle, its record), so it is built for four resident 512-thread blocks per SM.
__global__ void __launch_bounds__(512, 4) k_resolve(RefineArgs a, const int32_t* __restrict__ nearest,
                                                 const int32_t* __restrict__ rep_tri,
                                                 uint32_t* __restrict__ dist_bits, uint32_t* __restrict__ front,
                                                 uint32_t* __restrict__ back, float* __restrict__ sdf,
                                                 unsigned long long* __restrict__ bmask,
                                                 int32_t* __restrict__ blist, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ win_ray, int32_t* __restrict__ win_tri) {
    __shared__ unsigned long long smask[kMaxBricksPerTile];
    resolve_tile<kBX, kBY, kBZ>(a, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), nearest, rep_tri, dist_bits,
                                front, back, sdf, bmask, blist, count, win_ray, win_tri, 0, smask);
}

// ------------------------------------------------------------------ refine

// Persistent: warps take bricks from the work list until it is exhausted.  With kCull
// the bricks that refine_brick leaves to the per-ray launch go to dlist; with kRays
// the kernel is that launch and takes its bricks from dlist.
template <bool kTrack, int RPL, bool kCount, bool kCull, bool kRays = false>
__global__ void __launch_bounds__(kRefineThreads, refine_warps_per_sm<RPL>() * 32 / kRefineThreads) k_refine(RefineArgs a, const BvhHeader* __restrict__ hdr,
                                                              const BvhNode* __restrict__ nodes,
                                                              const BvhLeaf* __restrict__ leaves,
                                                              const int32_t* __restrict__ nearest,
                                                              const int32_t* __restrict__ rep_tri,
                                                              const unsigned long long* __restrict__ bmask,
                                                              const int32_t* __restrict__ blist,
                                                              int32_t* __restrict__ dlist,
                                                              uint32_t* __restrict__ count,
                                                              uint32_t* __restrict__ dist_bits,
                                                              uint32_t* __restrict__ front,
                                                              uint32_t* __restrict__ back, float* __restrict__ sdf,
                                                              rtsdf_counters* counters,
                                                              uint32_t* __restrict__ win_ray,
                                                              int32_t* __restrict__ win_tri) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmemT<RPL>& w = reinterpret_cast<WarpSmemT<RPL>*>(smem_raw)[warp];
    const int n_leaves = hdr->n_leaves;
    const int n_inner = n_leaves > 1 ? n_leaves - 1 : 1;
    const uint32_t nact = count[kRays ? 3 : 0];
    uint32_t n_hit = 0, n_fail = 0, n_ovf = 0;
    if (kCount) work_reset(w);
    while (true) {
        uint32_t wk = 0;
        if (lane == 0) wk = atomicAdd(count + (kRays ? 4 : 1), 1u);
        wk = __shfl_sync(0xffffffffu, wk, 0);
        if (wk >= nact) break;
        const int b = kRays ? dlist[wk] : blist[wk];
        const int bx = b % a.nbx, by = (b / a.nbx) % a.nby, bz = b / (a.nbx * a.nby);
        const bool deferred = refine_brick<kBX, kBY, kBZ, kTrack, RPL, kCount, kCull, kRays>(
            a, nodes, leaves, n_leaves, n_inner, nearest, rep_tri, bmask[b], bx, by, bz, dist_bits, front, back, sdf,
            win_ray, win_tri, w, n_hit, n_fail, n_ovf);
        if (deferred && lane == 0) dlist[atomicAdd(count + 3, 1u)] = b;
    }
    if (counters) {
        if (n_hit) atomicAdd(&counters->rays_hit, n_hit);
        if (n_fail) atomicAdd(&counters->rays_failed, n_fail);
    }
    if (kCount) work_flush(w, counters);
    if (lane == 0 && n_ovf) atomicAdd(count + 2, n_ovf);
}

template <bool kTrack, int RPL, bool kCount, bool kCull, bool kRays = false>
static rtsdf_status launch_refine_t(cudaStream_t s, const RefineArgs& a, const BvhHeader* hdr,
                                    const BvhNode* nodes, const BvhLeaf* leaves, const int32_t* nearest,
                                    const int32_t* rep_tri, const unsigned long long* bmask, const int32_t* blist,
                                    int32_t* dlist, uint32_t* count, uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf,
                                    rtsdf_counters* counters, uint32_t* win_ray, int32_t* win_tri) {
    const size_t smem = sizeof(WarpSmemT<RPL>) * (kRefineThreads / 32);
    static bool attr_set[64] = {};
    int dev = 0;
    RTSDF_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RTSDF_CUDA(cudaFuncSetAttribute(k_refine<kTrack, RPL, kCount, kCull, kRays>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = true;
    }
    k_refine<kTrack, RPL, kCount, kCull, kRays>
        <<<num_sms() * (refine_warps_per_sm<RPL>() * 32 / kRefineThreads), kRefineThreads, smem, s>>>(
            a, hdr, nodes, leaves, nearest, rep_tri, bmask, blist, dlist, count, dist_bits, front, back, sdf, counters,
            win_ray, win_tri);
    return RTSDF_OK;
}

static rtsdf_status launch_refine_kernel(bool track, bool count, bool cull, bool rays, int rpl, cudaStream_t s,
                                         const RefineArgs& a, const BvhHeader* hdr, const BvhNode* nodes,
                                         const BvhLeaf* leaves, const int32_t* nearest, const int32_t* rep_tri,
                                         const unsigned long long* bmask, const int32_t* blist, int32_t* dlist,
                                         uint32_t* wcount,
                                         uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf,
                                         rtsdf_counters* counters, uint32_t* win_ray, int32_t* win_tri) {
#define RTSDF_REFINE_CASE(T, R, N, C)                                                                           \
    if (track == T && rpl == R && count == N && cull == C && !rays)                                             \
        return launch_refine_t<T, R, N, C>(s, a, hdr, nodes, leaves, nearest, rep_tri, bmask, blist, dlist,     \
                                           wcount, dist_bits, front, back, sdf, counters, T ? win_ray : nullptr, \
                                           T ? win_tri : nullptr);                                               \
    if (!T && C && track == T && rpl == R && count == N && rays)                                                \
        return launch_refine_t<false, R, N, true, true>(s, a, hdr, nodes, leaves, nearest, rep_tri, bmask,      \
                                                        blist, dlist, wcount, dist_bits, front, back, sdf,      \
                                                        counters, nullptr, nullptr);
    RTSDF_REFINE_CASE(false, 2, false, false) RTSDF_REFINE_CASE(false, 4, false, false)
    RTSDF_REFINE_CASE(false, 8, false, false) RTSDF_REFINE_CASE(false, 16, false, false)
    RTSDF_REFINE_CASE(true, 2, false, false) RTSDF_REFINE_CASE(true, 4, false, false)
    RTSDF_REFINE_CASE(true, 8, false, false) RTSDF_REFINE_CASE(true, 16, false, false)
    RTSDF_REFINE_CASE(false, 2, true, false) RTSDF_REFINE_CASE(false, 4, true, false)
    RTSDF_REFINE_CASE(false, 8, true, false) RTSDF_REFINE_CASE(false, 16, true, false)
    RTSDF_REFINE_CASE(false, 2, false, true) RTSDF_REFINE_CASE(false, 4, false, true)
    RTSDF_REFINE_CASE(false, 8, false, true) RTSDF_REFINE_CASE(false, 16, false, true)
    RTSDF_REFINE_CASE(false, 2, true, true) RTSDF_REFINE_CASE(false, 4, true, true)
    RTSDF_REFINE_CASE(false, 8, true, true) RTSDF_REFINE_CASE(false, 16, true, true)
#undef RTSDF_REFINE_CASE
    return RTSDF_EINVAL;
}

// Masked voxels (set bits over all bricks) and walks that overflowed, to the counters.
__global__ void k_refine_report(const uint32_t* __restrict__ count, const unsigned long long* __restrict__ bmask,
                                size_t nb, rtsdf_counters* counters) {
    uint32_t n = 0;
    for (size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (size_t)gridDim.x * blockDim.x)
        n += __popcll(bmask[b]);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&counters->masked_voxels, n);
    if (blockIdx.x == 0 && threadIdx.x == 0 && count[2]) atomicAdd(&counters->stack_overflow, count[2]);
}

rtsdf_status refine(const rtsdf_grid& gh, int32_t T, const void* bvh, const int32_t* nearest, const int32_t* rep_tri,
                    const rtsdf_refine_params& p, uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf, void* ws,
                    rtsdf_counters* counters, uint32_t* win_ray, int32_t* win_tri, const rtsdf_grid* coarse,
                    int ratio, cudaStream_t s) {
    RefineArgs a;
    a.g = to_dev(gh);
    a.T = T;
    a.mask2 = p.mask_vox * p.mask_vox;
    a.beta = p.beta_vox;
    a.empty_dist = (float)(gh.nx + gh.ny + gh.nz);
    a.R = p.rays_per_voxel;
    a.tmax = p.max_ray_vox;
    a.k0 = p.key[0];
    a.k1 = p.key[1];
    a.frame = p.frame_index;
    a.scene = p.scene_id;
    a.accumulate = p.accumulate;
    a.alpha = p.decay_alpha;
    a.one_minus_alpha = 1.0f - p.decay_alpha;
    a.fallback = p.sign_fallback;
    a.ratio = coarse ? ratio : 1;
    a.cnx = coarse ? coarse->nx : gh.nx;
    a.cny = coarse ? coarse->ny : gh.ny;
    a.cnz = coarse ? coarse->nz : gh.nz;
    a.nbx = (gh.nx + kBX - 1) / kBX;
    a.nby = (gh.ny + kBY - 1) / kBY;
    a.nbz = (gh.nz + kBZ - 1) / kBZ;
    a.per_ray = 0;
    RefineWs w;
    refine_ws_layout(gh, static_cast<char*>(ws), &w);
    const auto* hdr = static_cast<const BvhHeader*>(bvh);
    const auto* nodes = reinterpret_cast<const BvhNode*>(static_cast<const char*>(bvh) + bvh_nodes_offset());
    const auto* leaves = reinterpret_cast<const BvhLeaf*>(static_cast<const char*>(bvh) + bvh_leaves_offset(T));
    a.tv = reinterpret_cast<const TriVox*>(static_cast<const char*>(bvh) + bvh_tris_offset(T));
    RTSDF_CUDA(cudaMemsetAsync(w.count, 0, 32, s));
    const dim3 rgrid((gh.nx + 31) / 32, (gh.ny + 3) / 4, (gh.nz + 3) / 4);
    const bool track = win_ray != nullptr;
    k_resolve<<<rgrid, 512, 0, s>>>(a, nearest, rep_tri, dist_bits, front, back, sdf, w.bmask, w.blist, w.count,
                                    track ? win_ray : nullptr, track ? win_tri : nullptr);
    RTSDF_LAUNCHED();
    const int rpl = a.R <= 2 ? 2 : (a.R <= 4 ? 4 : (a.R <= 8 ? 8 : 16));  // one ray group for up to rpl rays
    // work counting: only untracked calls that pass counters and ask for it
    const bool count_work = !track && counters != nullptr && p.count_work != 0;
    // coarse grids (many triangles within a brick's reach) take the culling instantiation;
    // tracked calls (the adjoint's forward) keep the plain one
    const double est = staged_estimate(T, gh.nx, gh.ny, gh.nz, a.tmax, kBX, kBY, kBZ);
    const bool cull = !track && est >= kCullEstimate;
    a.per_ray = cull && est >= per_ray_estimate(a.R) ? 1 : 0;
    RTSDF_TRY(launch_refine_kernel(track, count_work, cull, false, rpl, s, a, hdr, nodes, leaves, nearest, rep_tri,
                                   w.bmask, w.blist, w.dlist, w.count, dist_bits, front, back, sdf, counters, win_ray,
                                   win_tri));
    RTSDF_LAUNCHED();
    if (a.per_ray) {  // the bricks the first launch left to the per-ray walk
        RTSDF_TRY(launch_refine_kernel(track, count_work, cull, true, rpl, s, a, hdr, nodes, leaves, nearest, rep_tri,
                                       w.bmask, w.blist, w.dlist, w.count, dist_bits, front, back, sdf, counters,
                                       win_ray, win_tri));
        RTSDF_LAUNCHED();
    }
    if (counters) {
        k_refine_report<<<num_sms(), 256, 0, s>>>(w.count, w.bmask, nbricks(gh), counters);
        RTSDF_LAUNCHED();
    }
    return RTSDF_OK;
}

}  // namespace rtsdf
