// Coarse field, ray mask and ray-sampled refinement (Sec. 2.1-2.3).
//
//  k_resolve: one thread per voxel, blocks of 32x4x4 voxels = 8 bricks of 4^3.
//             Coarse distance u_c to the representative triangle of the flooded
//             seed; unmasked voxels get their final value (u_c - beta); masked
//             voxels initialise their refine state.  Per brick a 64-bit mask of
//             its masked voxels is assembled from warp ballots, and bricks with
//             any masked voxel are appended to a work list.
//  k_refine:  persistent warp-per-voxel-batch refinement, one 4^3 brick per
//             64-thread CTA.  Warp 0 walks the BVH once for the whole brick with
//             the box every ray of the brick stays inside (voxel centres grown
//             by the ray length) and stages the overlapping triangles in shared
//             memory; every thread owns one masked voxel and tests its rays
//             against the staged triangles after a bounding-sphere cull of the
//             (voxel, triangle) pair.  The closest hit of each ray (ties to the
//             lower triangle id) lowers the voxel's distance and adds one
//             front/back vote; the thread then writes the accumulated state and
//             the signed value.  Staging runs in rounds when a brick has more
//             candidates than the buffer holds.
#include <float.h>

#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

constexpr int kB = 4;                // brick edge (voxels)
constexpr int kRefineThreads = 64;   // independent warps, one brick each
constexpr int kListCap = 512;        // staged leaves per warp and round
constexpr int kStackCapW = 256;      // traversal stack per warp (entries)
constexpr int kRaysPerLane = 8;      // rays of a voxel per group (one lane per voxel)
constexpr int kFilterBatch = 4;      // staged triangles filtered per enqueue
constexpr int kQueueCap = 32 + 32 * 8 * kFilterBatch;  // queued ray/triangle items per warp

struct RefineWs {
    uint32_t* count;            // [0] active bricks, [1] work counter, [2] walks that overflowed
    unsigned long long* bmask;  // per brick: bit (lz*16 + ly*4 + lx) set for masked voxels
    int32_t* blist;             // active bricks
};

static size_t nbricks(const rtsdf_grid& g) {
    return (size_t)((g.nx + kB - 1) / kB) * ((g.ny + kB - 1) / kB) * ((g.nz + kB - 1) / kB);
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
    if (w) {
        w->count = reinterpret_cast<uint32_t*>(c);
        w->bmask = reinterpret_cast<unsigned long long*>(m);
        w->blist = reinterpret_cast<int32_t*>(l);
    }
    return off;
}

size_t refine_workspace(const rtsdf_grid& g) { return refine_ws_layout(g, nullptr, nullptr); }

struct RefineArgs {
    GridD g;
    const float* verts;
    int V;
    const int32_t* tris;
    float mask2;
    float beta;
    float empty_dist;
    int R;
    float tmax;
    uint32_t k0, k1, frame, scene;
    int accumulate, fallback;
    int nbx, nby, nbz;
};

// ------------------------------------------------------------------ resolve

__global__ void __launch_bounds__(512) k_resolve(RefineArgs a, const int32_t* __restrict__ nearest,
                                                 const int32_t* __restrict__ rep_tri,
                                                 uint32_t* __restrict__ dist_bits, uint32_t* __restrict__ front,
                                                 uint32_t* __restrict__ back, float* __restrict__ sdf,
                                                 unsigned long long* __restrict__ bmask,
                                                 int32_t* __restrict__ blist, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ win_ray, int32_t* __restrict__ win_tri) {
    __shared__ unsigned long long smask[8];
    const int tx = threadIdx.x & 31, ty = (threadIdx.x >> 5) & 3, tz = threadIdx.x >> 7;
    const int i = blockIdx.x * 32 + tx, j = blockIdx.y * kB + ty, k = blockIdx.z * kB + tz;
    if (threadIdx.x < 8) smask[threadIdx.x] = 0ull;
    __syncthreads();
    bool masked = false;
    if (i < a.g.nx && j < a.g.ny && k < a.g.nz) {
        const int64_t lin = ((int64_t)k * a.g.ny + j) * a.g.nx + i;
        const int32_t s = __ldg(nearest + lin);
        int32_t rep = -1;
        int si = 0, sj = 0, sk = 0;
        if (s != RTSDF_EMPTY) {
            si = s & 1023;
            sj = (s >> 10) & 1023;
            sk = (s >> 20) & 1023;
            rep = __ldg(rep_tri + ((int64_t)sk * a.g.ny + sj) * a.g.nx + si);
        }
        float uc = a.empty_dist;
        float3 A, B, C;
        if (rep >= 0 && load_tri(a.verts, a.V, a.tris, rep, a.g, A, B, C)) {
            const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
            uc = sqrtf(closest_d2(p, A, B, C));
            const int dx = i - si, dy = j - sj, dz = k - sk;
            masked = (float)(dx * dx + dy * dy + dz * dz) <= a.mask2;
        }
        // winner record (tracked calls): the coarse source holds a voxel's distance
        // when the voxel is unmasked, starts fresh, or its coarse distance is lower
        bool coarse_wins = true;
        if (!masked) {
            sdf[lin] = uc - a.beta;
        } else {
            const uint32_t ub = __float_as_uint(uc);
            if (a.accumulate) {
                const uint32_t old = dist_bits[lin];
                coarse_wins = ub < old;
                dist_bits[lin] = min(old, ub);
            } else {
                dist_bits[lin] = ub;
                front[lin] = 0u;
                back[lin] = 0u;
            }
        }
        if (win_ray && coarse_wins) {
            win_ray[lin] = 0xFFFFFFFFu;
            win_tri[lin] = -1;
        }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, masked);
    if (tx == 0 && bal) {
        const int shift = (tz * kB + ty) * kB;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned long long nib = (bal >> (4 * b)) & 0xFu;
            if (nib) atomicOr(&smask[b], nib << shift);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int bx = blockIdx.x * 8 + threadIdx.x;
        const bool valid = threadIdx.x < 8 && bx < a.nbx;
        const unsigned long long m = valid ? smask[threadIdx.x] : 0ull;
        const int64_t b = ((int64_t)blockIdx.z * a.nby + blockIdx.y) * a.nbx + bx;
        if (valid) bmask[b] = m;
        const uint32_t act = __ballot_sync(0xffffffffu, m != 0ull);
        uint32_t base = 0;
        if (threadIdx.x == 0 && act) base = atomicAdd(count, (uint32_t)__popc(act));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (m) blist[base + __popc(act & ((1u << threadIdx.x) - 1u))] = (int32_t)b;
    }
}

// ------------------------------------------------------------------ refine

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
// the new list length; `sp` is the stack depth.
__device__ __forceinline__ int walk_and_stage(const BvhNode* __restrict__ nodes, int n_inner, int n_leaves,
                                              float3 qlo, float3 qhi, float ext2, int* stack, int& sp,
                                              int* list, int nc, bool& overflow) {
    const int lane = threadIdx.x & 31;
    int guard = 0;
    while (sp > 0 && nc <= kListCap - 64) {
        if (++guard > n_inner + 64) {  // a well-formed tree is exhausted long before
            overflow = true;
            sp = 0;
            break;
        }
        const int take = min(sp, 32);
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

// Per-warp shared state of k_refine.
struct WarpSmem {
    int list[kListCap];             // staged leaves
    int stack[kStackCapW];
    uint32_t queue[kQueueCap];      // (list index << 8) | (slot << 3) | ray
    int qn;                         // queued items
    float4 origin[32];              // voxel centres of the pass's slots
    float4 dir[8][32];              // ray directions of the group, [ray][slot]
    unsigned long long key[8][32];  // closest hit: (t bits << 32) | (id << 1) | front
};

// Exact Moller-Trumbore test of one queued (voxel, ray, triangle) item; the
// closest hit per ray (ties to the lower id) is kept with a 64-bit atomicMin.
__device__ __forceinline__ void run_item(WarpSmem& w, const BvhLeaf* __restrict__ leaves, uint32_t item,
                                         float tmax) {
    const int c = (int)(item >> 8), slot = (int)((item >> 3) & 31u), r = (int)(item & 7u);
    const float4 of = w.origin[slot], df = w.dir[r][slot];
    const float3 o = make_float3(of.x, of.y, of.z), d = make_float3(df.x, df.y, df.z);
    const BvhLeaf* L = leaves + w.list[c];
    const float4 v0 = __ldg(&L->v0), e1f = __ldg(&L->e1), e2f = __ldg(&L->e2);
    const float3 A = make_float3(v0.x, v0.y, v0.z);
    const float3 e1 = make_float3(e1f.x, e1f.y, e1f.z), e2 = make_float3(e2f.x, e2f.y, e2f.z);
    float t;
    bool front;
    if (ray_tri(o, d, A, e1, e2, tmax, t, front)) {
        const uint32_t id = (uint32_t)__float_as_int(v0.w);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)((id << 1) | (front ? 1u : 0u));
        atomicMin(&w.key[r][slot], key);
    }
}

// Which of this lane's rays can hit the triangle of `leaf`: the (voxel, triangle)
// pair must be within reach of the bounding sphere; each ray's line must pass
// within rho of the sphere centre with the centre at most rho behind the origin
// (off the rho-sphere by more than rho*sqrt(2) that is exactly tc >= sqrt(dd -
// rho^2); nearer, tc >= -rho is kept, a superset); and the ray must head for the
// triangle's plane and cross it within the ray length.  All margins exceed the
// FP32 rounding of both sides, so no triangle the exact test accepts is dropped.
__device__ __forceinline__ uint32_t filter_rays(const BvhLeaf* __restrict__ leaf, float3 o, uint32_t okm,
                                                const float2* dx2, const float2* dy2, const float2* dz2,
                                                float tmax) {
    const float4 sph = __ldg(&leaf->sph);
    const float dcx = sph.x - o.x, dcy = sph.y - o.y, dcz = sph.z - o.z;
    const float dd = __fmaf_rn(dcx, dcx, __fmaf_rn(dcy, dcy, dcz * dcz));
    const float reach = sph.w + tmax;
    if (!okm || dd > reach * reach) return 0u;
    const float4 pl = __ldg(&leaf->pln);
    const float rho = sph.w;
    const float rho2 = rho * rho;
    const float thr = dd > 2.0f * rho2 ? __fsqrt_rn(dd - rho2) * 0.999999f - 1e-4f : -rho;
    const float sd = pl.w - __fmaf_rn(pl.x, o.x, __fmaf_rn(pl.y, o.y, pl.z * o.z));
    const float eps = 2e-3f + 2e-6f * fabsf(pl.w);
    const float asd = fabsf(sd);
    const float2 cx2 = make_float2(dcx, dcx), cy2 = make_float2(dcy, dcy), cz2 = make_float2(dcz, dcz);
    const float2 nx2 = make_float2(pl.x, pl.x), ny2 = make_float2(pl.y, pl.y), nz2 = make_float2(pl.z, pl.z);
    uint32_t pm = 0;
#pragma unroll
    for (int r = 0; r < kRaysPerLane / 2; ++r) {
        const float2 tc = __ffma2_rn(cx2, dx2[r], __ffma2_rn(cy2, dy2[r], __fmul2_rn(cz2, dz2[r])));
        const float2 dn = __ffma2_rn(nx2, dx2[r], __ffma2_rn(ny2, dy2[r], __fmul2_rn(nz2, dz2[r])));
        const bool ok0 = tc.x >= thr && sd * dn.x > -eps && asd <= __fmaf_rn(tmax, fabsf(dn.x), eps);
        const bool ok1 = tc.y >= thr && sd * dn.y > -eps && asd <= __fmaf_rn(tmax, fabsf(dn.y), eps);
        pm |= ((ok0 ? 1u : 0u) << (2 * r)) | ((ok1 ? 1u : 0u) << (2 * r + 1));
    }
    return pm & okm;
}

// One warp per brick; lane l owns voxel slot (pass*32 + l) and up to 8 rays of it
// per group.  For every staged triangle the lane culls the (voxel, triangle) pair
// by the triangle's bounding sphere grown by the ray length, then each ray by the
// distance of the sphere's centre to the ray's line (and the side it lies on).
// Surviving (voxel, ray, triangle) items are queued in shared memory and run
// through the exact ray/triangle test 32 at a time, so the expensive test does
// not diverge.  Both filters are conservative (their margins exceed FP32 rounding
// of the exact test), so they never drop a triangle the exact test accepts; they
// may use fused multiply-adds because they decide nothing the oracle decides.
template <bool kTrack>
__global__ void __launch_bounds__(kRefineThreads, 8) k_refine(RefineArgs a, const BvhHeader* __restrict__ hdr,
                                                              const BvhNode* __restrict__ nodes,
                                                              const BvhLeaf* __restrict__ leaves,
                                                              const int32_t* __restrict__ nearest,
                                                              const int32_t* __restrict__ rep_tri,
                                                              const unsigned long long* __restrict__ bmask,
                                                              const int32_t* __restrict__ blist,
                                                              uint32_t* __restrict__ count,
                                                              uint32_t* __restrict__ dist_bits,
                                                              uint32_t* __restrict__ front,
                                                              uint32_t* __restrict__ back, float* __restrict__ sdf,
                                                              rtsdf_counters* counters,
                                                              uint32_t* __restrict__ win_ray,
                                                              int32_t* __restrict__ win_tri) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem& w = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
    const int n_leaves = hdr->n_leaves;
    const int n_inner = n_leaves > 1 ? n_leaves - 1 : 1;
    const uint32_t nact = count[0];
    uint32_t n_hit = 0, n_fail = 0, n_ovf = 0;
    const float ext = a.tmax * 1.00001f + 1e-3f;

    while (true) {
        uint32_t wk = 0;
        if (lane == 0) wk = atomicAdd(count + 1, 1u);
        wk = __shfl_sync(0xffffffffu, wk, 0);
        if (wk >= nact) break;
        const int b = blist[wk];
        const int bx = b % a.nbx, by = (b / a.nbx) % a.nby, bz = b / (a.nbx * a.nby);
        const unsigned long long m = bmask[b];
        const int nm = __popcll(m);
        // every ray of the brick stays inside its voxel centres' box grown by the ray length
        const float3 qlo = make_float3((float)(bx * kB) + 0.5f, (float)(by * kB) + 0.5f, (float)(bz * kB) + 0.5f);
        const float3 qhi = make_float3((float)(bx * kB + kB - 1) + 0.5f, (float)(by * kB + kB - 1) + 0.5f,
                                       (float)(bz * kB + kB - 1) + 0.5f);
        bool overflow = false;
        // walk once for the whole brick; the list is reused by every pass and ray
        // group unless it overflowed, in which case each pass walks again in rounds
        int sp0 = 0;
        if (n_leaves > 0) {
            if (lane == 0) w.stack[0] = 0;
            sp0 = 1;
        }
        __syncwarp();
        const int nc_all = walk_and_stage(nodes, n_inner, n_leaves, qlo, qhi, ext * ext, w.stack, sp0, w.list, 0,
                                          overflow);
        const bool complete = sp0 == 0;
        for (int pass = 0; pass * 32 < nm; ++pass) {
            const int slot = pass * 32 + lane;
            const bool mine = slot < nm;
            int lin = 0;
            float3 o = make_float3(0.f, 0.f, 0.f);
            if (mine) {
                // position of the slot-th set bit of the brick mask
                unsigned long long mm = m;
                int skip = slot;
                const int lo_cnt = __popc((uint32_t)mm);
                if (skip >= lo_cnt) {
                    skip -= lo_cnt;
                    mm &= 0xffffffff00000000ull;
                }
                for (int c = 0; c < skip; ++c) mm &= mm - 1ull;
                const int bit = __ffsll((long long)mm) - 1;
                const int i = bx * kB + (bit & 3), j = by * kB + ((bit >> 2) & 3), k = bz * kB + (bit >> 4);
                lin = (int)(((int64_t)k * a.g.ny + j) * a.g.nx + i);
                o = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
            }
            w.origin[lane] = make_float4(o.x, o.y, o.z, 0.f);
            uint32_t vbest = 0xffffffffu, vfront = 0, vback = 0;
            // tracked: this call's winning ray, ordered by (t, triangle id), first ray on ties
            unsigned long long wkey = ~0ull;
            uint32_t wray = 0xFFFFFFFFu;
            for (int r0 = 0; r0 < a.R; r0 += kRaysPerLane) {
                float3 dir[kRaysPerLane];
                uint32_t okm = 0;
#pragma unroll
                for (int r = 0; r < kRaysPerLane; ++r) {
                    const int ray = r0 + r;
                    dir[r] = make_float3(0.f, 0.f, 1.f);
                    if (mine && ray < a.R) {
                        if (sphere_dir((uint32_t)lin, a.frame * (uint32_t)a.R + (uint32_t)ray, a.scene, a.k0, a.k1,
                                       dir[r]))
                            okm |= 1u << r;
                        else
                            ++n_fail;
                    }
                    w.dir[r][lane] = make_float4(dir[r].x, dir[r].y, dir[r].z, 0.f);
                    w.key[r][lane] = ~0ull;
                }
                float2 dx2[kRaysPerLane / 2], dy2[kRaysPerLane / 2], dz2[kRaysPerLane / 2];
#pragma unroll
                for (int r = 0; r < kRaysPerLane / 2; ++r) {
                    dx2[r] = make_float2(dir[2 * r].x, dir[2 * r + 1].x);
                    dy2[r] = make_float2(dir[2 * r].y, dir[2 * r + 1].y);
                    dz2[r] = make_float2(dir[2 * r].z, dir[2 * r + 1].z);
                }
                int sp = 0;
                if (!complete && n_leaves > 0) {
                    if (lane == 0) w.stack[0] = 0;
                    sp = 1;
                }
                __syncwarp();
                bool first = true;
                while (first || sp > 0) {
                    first = false;
                    const int nc = complete ? nc_all
                                            : walk_and_stage(nodes, n_inner, n_leaves, qlo, qhi, ext * ext, w.stack,
                                                             sp, w.list, 0, overflow);
                    if (lane == 0) w.qn = 0;
                    __syncwarp();
                    for (int c0 = 0; c0 < nc; c0 += kFilterBatch) {
                        // filter kFilterBatch staged triangles (independent work), then each lane
                        // that has survivors claims queue slots with one shared atomic
                        uint32_t pm4 = 0;  // bit (j * 8 + r): ray r vs triangle c0 + j
#pragma unroll
                        for (int j = 0; j < kFilterBatch; ++j) {
                            const int c = c0 + j;
                            if (c < nc) pm4 |= filter_rays(leaves + w.list[c], o, okm, dx2, dy2, dz2, a.tmax) << (8 * j);
                        }
                        if (pm4) {
                            int pos = atomicAdd(&w.qn, __popc(pm4));
                            while (pm4) {
                                const int bit = __ffs(pm4) - 1;
                                pm4 &= pm4 - 1u;
                                w.queue[pos++] =
                                    ((uint32_t)(c0 + (bit >> 3)) << 8) | ((uint32_t)lane << 3) | (uint32_t)(bit & 7);
                            }
                        }
                        __syncwarp();
                        int qn = w.qn;
                        if (qn >= 32) {
                            while (qn >= 32) {
                                run_item(w, leaves, w.queue[qn - 32 + lane], a.tmax);
                                qn -= 32;
                            }
                            __syncwarp();
                            if (lane == 0) w.qn = qn;
                            __syncwarp();
                        }
                    }
                    {
                        const int qn = w.qn;
                        if (lane < qn) run_item(w, leaves, w.queue[lane], a.tmax);
                        __syncwarp();
                    }
                    __syncwarp();
                    __syncwarp();
                }
                // closest hits of this lane's rays
#pragma unroll
                for (int r = 0; r < kRaysPerLane; ++r) {
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
                    const int32_t s = nearest[lin];
                    const int64_t sl2 =
                        ((int64_t)((s >> 20) & 1023) * a.g.ny + ((s >> 10) & 1023)) * a.g.nx + (s & 1023);
                    float3 A, B, C;
                    load_tri(a.verts, a.V, a.tris, rep_tri[sl2], a.g, A, B, C);
                    const float3 n = cross3(sub3(B, A), sub3(C, A));
                    neg = dot3(sub3(o, A), n) < 0.0f;
                }
                const float df = __uint_as_float(d);
                sdf[lin] = neg ? -df : df;
            }
            __syncwarp();
        }
        n_ovf += overflow ? 1u : 0u;
    }
    if (counters) {
        if (n_hit) atomicAdd(&counters->rays_hit, n_hit);
        if (n_fail) atomicAdd(&counters->rays_failed, n_fail);
    }
    if (lane == 0 && n_ovf) atomicAdd(count + 2, n_ovf);
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

rtsdf_status refine(const rtsdf_grid& gh, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                    const void* bvh, const int32_t* nearest, const int32_t* rep_tri, const rtsdf_refine_params& p,
                    uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf, void* ws,
                    rtsdf_counters* counters, uint32_t* win_ray, int32_t* win_tri, cudaStream_t s) {
    RefineArgs a;
    a.g = to_dev(gh);
    a.verts = verts;
    a.V = V;
    a.tris = tris;
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
    a.fallback = p.sign_fallback;
    a.nbx = (gh.nx + kB - 1) / kB;
    a.nby = (gh.ny + kB - 1) / kB;
    a.nbz = (gh.nz + kB - 1) / kB;
    RefineWs w;
    refine_ws_layout(gh, static_cast<char*>(ws), &w);
    const auto* hdr = static_cast<const BvhHeader*>(bvh);
    const auto* nodes = reinterpret_cast<const BvhNode*>(static_cast<const char*>(bvh) + bvh_nodes_offset());
    const auto* leaves = reinterpret_cast<const BvhLeaf*>(static_cast<const char*>(bvh) + bvh_leaves_offset(T));
    RTSDF_CUDA(cudaMemsetAsync(w.count, 0, 16, s));
    const dim3 rgrid((gh.nx + 31) / 32, a.nby, a.nbz);
    const bool track = win_ray != nullptr;
    k_resolve<<<rgrid, 512, 0, s>>>(a, nearest, rep_tri, dist_bits, front, back, sdf, w.bmask, w.blist, w.count,
                                    track ? win_ray : nullptr, track ? win_tri : nullptr);
    RTSDF_LAUNCHED();
    const size_t smem = sizeof(WarpSmem) * (kRefineThreads / 32);
    static bool attr_set[64][2] = {};
    int dev = 0;
    RTSDF_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev][track]) {
        RTSDF_CUDA(cudaFuncSetAttribute(track ? k_refine<true> : k_refine<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev][track] = true;
    }
    if (track)
        k_refine<true><<<num_sms() * 8, kRefineThreads, smem, s>>>(a, hdr, nodes, leaves, nearest, rep_tri, w.bmask,
                                                                 w.blist, w.count, dist_bits, front, back, sdf,
                                                                 counters, win_ray, win_tri);
    else
        k_refine<false><<<num_sms() * 8, kRefineThreads, smem, s>>>(a, hdr, nodes, leaves, nearest, rep_tri, w.bmask,
                                                                  w.blist, w.count, dist_bits, front, back, sdf,
                                                                  counters, nullptr, nullptr);
    RTSDF_LAUNCHED();
    if (counters) {
        k_refine_report<<<num_sms(), 256, 0, s>>>(w.count, w.bmask, nbricks(gh), counters);
        RTSDF_LAUNCHED();
    }
    return RTSDF_OK;
}

}  // namespace rtsdf
