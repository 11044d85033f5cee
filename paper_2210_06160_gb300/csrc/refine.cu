// Coarse field, ray mask and ray-sampled refinement (Sec. 2.1-2.3).
//
//  k_resolve:  one thread per voxel.  Coarse distance u_c to the representative
//              triangle of the flooded seed; unmasked voxels get their final
//              value (u_c - beta); masked voxels initialise their refine state
//              and are appended to a compacted list (warp ballot + one atomic
//              per warp).
//  k_trace:    persistent; warps take 32 (voxel, ray) items at a time from a
//              global counter.  Each lane draws its Philox direction and walks
//              the BVH (stack traversal, nearest child first, boxes clipped to
//              the closest hit so far); per voxel, the closest hits are reduced
//              in-warp when R divides 32, else merged with atomics.
//  k_finalize: signs the masked voxels from their front/back votes.
#include <float.h>

#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

struct RefineWs {
    int32_t* list;
    uint32_t* count;    // [0] masked voxels, [1] work counter
};

static size_t refine_ws_layout(const rtsdf_grid& g, char* base, RefineWs* w) {
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    size_t off = 0;
    char* c = base;
    off += 256;
    char* l = base ? base + off : nullptr;
    off += align_up(4 * nvox, 256);
    if (w) {
        w->count = reinterpret_cast<uint32_t*>(c);
        w->list = reinterpret_cast<int32_t*>(l);
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
};

__global__ void __launch_bounds__(256) k_resolve(RefineArgs a, const int32_t* __restrict__ nearest,
                                                 const int32_t* __restrict__ rep_tri, uint32_t* __restrict__ dist_bits,
                                                 uint32_t* __restrict__ front, uint32_t* __restrict__ back,
                                                 float* __restrict__ sdf, int32_t* __restrict__ list,
                                                 uint32_t* __restrict__ count) {
    const int64_t nvox = (int64_t)a.g.nx * a.g.ny * a.g.nz;
    const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool masked = false;
    if (lin < nvox) {
        const int64_t plane = (int64_t)a.g.nx * a.g.ny;
        const int k = (int)(lin / plane), rem = (int)(lin - (int64_t)k * plane);
        const int j = rem / a.g.nx, i = rem - j * a.g.nx;
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
        if (!masked) {
            sdf[lin] = uc - a.beta;
        } else {
            const uint32_t ub = __float_as_uint(uc);
            if (a.accumulate) {
                dist_bits[lin] = min(dist_bits[lin], ub);
            } else {
                dist_bits[lin] = ub;
                front[lin] = 0u;
                back[lin] = 0u;
            }
        }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, masked);
    if (bal == 0u) return;
    const uint32_t lane = lane_id();
    uint32_t base = 0;
    if (lane == (uint32_t)(__ffs(bal) - 1)) base = atomicAdd(count, (uint32_t)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
    if (masked) list[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)lin;
}

struct Hit {
    float t;
    int id;
    bool front;
};

__device__ __forceinline__ bool slab(float4 lo, float4 hi, float3 o, float3 inv, float tclip, float& tnear) {
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tclip));
    tnear = tn;
    return tn <= tf;
}

constexpr int kStack = 64;

__device__ __forceinline__ void leaf_test(const BvhLeaf* __restrict__ leaves, int j, float3 o, float3 d, float tmax,
                                          Hit& best, float& tclip) {
    const float4 v0 = __ldg(&leaves[j].v0), e1 = __ldg(&leaves[j].e1), e2 = __ldg(&leaves[j].e2);
    const int id = __float_as_int(v0.w);
    float t;
    bool f;
    if (ray_tri(o, d, make_float3(v0.x, v0.y, v0.z), make_float3(e1.x, e1.y, e1.z), make_float3(e2.x, e2.y, e2.z),
                tmax, t, f)) {
        if (t < best.t || (t == best.t && id < best.id)) {
            best.t = t;
            best.id = id;
            best.front = f;
            tclip = t;
        }
    }
}

// Closest hit among all triangles with 0 < t <= tmax (ties -> lower id).
// n_inner: number of inner nodes (n_leaves - 1, at least 1).  Every node is
// entered at most once per ray in a well-formed tree; the loop is additionally
// bounded and index-checked so that a malformed buffer ends the walk (flagged as
// overflow) instead of reading out of bounds or spinning.
__device__ __forceinline__ Hit trace_ray(const BvhNode* __restrict__ nodes, const BvhLeaf* __restrict__ leaves,
                                         int n_inner, int n_leaves, float3 o, float3 d, float tmax, bool& overflow) {
    Hit best{FLT_MAX, 0x7fffffff, false};
    const float3 inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int stack[kStack];
    int sp = 0, cur = 0;
    float tclip = tmax;
    for (int guard = 0; guard <= n_inner; ++guard) {
        if (cur < 0 || cur >= n_inner) { overflow = true; break; }
        const BvhNode* nd = nodes + cur;
        const float4 lo0 = __ldg(&nd->lo0), hi0 = __ldg(&nd->hi0), lo1 = __ldg(&nd->lo1), hi1 = __ldg(&nd->hi1);
        const int c0 = __float_as_int(lo0.w), c1 = __float_as_int(hi0.w);
        float tn0, tn1;
        bool h0 = slab(lo0, hi0, o, inv, tclip, tn0);
        bool h1 = slab(lo1, hi1, o, inv, tclip, tn1);
        if (h0 && c0 < 0) { if (~c0 < n_leaves) leaf_test(leaves, ~c0, o, d, tmax, best, tclip); h0 = false; }
        if (h1 && c1 < 0) { if (~c1 < n_leaves) leaf_test(leaves, ~c1, o, d, tmax, best, tclip); h1 = false; }
        int next;
        if (h0 && h1) {
            const bool first0 = tn0 <= tn1;
            if (sp < kStack) stack[sp++] = first0 ? c1 : c0; else overflow = true;
            next = first0 ? c0 : c1;
        } else if (h0) {
            next = c0;
        } else if (h1) {
            next = c1;
        } else {
            if (sp == 0) break;
            next = stack[--sp];
        }
        cur = next;
    }
    return best;
}

__global__ void __launch_bounds__(256) k_trace(RefineArgs a, const BvhHeader* __restrict__ hdr,
                                               const BvhNode* __restrict__ nodes, const BvhLeaf* __restrict__ leaves,
                                               const int32_t* __restrict__ list, uint32_t* __restrict__ count,
                                               uint32_t* __restrict__ dist_bits, uint32_t* __restrict__ front,
                                               uint32_t* __restrict__ back, rtsdf_counters* counters) {
    const int n_leaves = hdr->n_leaves;
    const uint64_t total = (uint64_t)count[0] * (uint64_t)a.R;
    const uint32_t lane = lane_id();
    const bool grouped = (32 % a.R) == 0;  // a voxel's R rays sit in one warp chunk
    uint32_t n_hit = 0, n_fail = 0, n_ovf = 0;
    while (true) {
        uint64_t base = 0;
        if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(count + 2), 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const uint64_t item = base + lane;
        const bool active = item < total;
        Hit h{FLT_MAX, 0x7fffffff, false};
        int lin = 0;
        if (active) {
            const uint32_t li = (uint32_t)(item / (uint32_t)a.R), r = (uint32_t)(item % (uint32_t)a.R);
            lin = __ldg(list + li);
            const int64_t plane = (int64_t)a.g.nx * a.g.ny;
            const int k = (int)(lin / plane), rem = (int)(lin - (int64_t)k * plane);
            const int j = rem / a.g.nx, i = rem - j * a.g.nx;
            const float3 o = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
            float3 d;
            if (!sphere_dir((uint32_t)lin, a.frame * (uint32_t)a.R + r, a.scene, a.k0, a.k1, d)) {
                ++n_fail;
            } else if (n_leaves > 0) {
                bool ovf = false;
                h = trace_ray(nodes, leaves, n_leaves > 1 ? n_leaves - 1 : 1, n_leaves, o, d, a.tmax, ovf);
                n_ovf += ovf;
            }
        }
        const bool hit = h.id != 0x7fffffff;
        n_hit += hit;
        if (grouped) {
            // reduce the R lanes of each voxel: min t, front and back vote counts
            uint32_t tb = hit ? __float_as_uint(h.t) : 0xffffffffu;
            uint32_t nf = (hit && h.front) ? 1u : 0u, nb = (hit && !h.front) ? 1u : 0u;
            for (int o2 = 1; o2 < a.R; o2 <<= 1) {
                tb = min(tb, __shfl_xor_sync(0xffffffffu, tb, o2));
                nf += __shfl_xor_sync(0xffffffffu, nf, o2);
                nb += __shfl_xor_sync(0xffffffffu, nb, o2);
            }
            if (active && (lane % (uint32_t)a.R) == 0) {
                if (tb != 0xffffffffu) dist_bits[lin] = min(dist_bits[lin], tb);
                front[lin] += nf;
                back[lin] += nb;
            }
        } else if (active && hit) {
            atomicMin(dist_bits + lin, __float_as_uint(h.t));
            atomicAdd(h.front ? front + lin : back + lin, 1u);
        }
    }
    if (counters) {
        if (n_hit) atomicAdd(&counters->rays_hit, n_hit);
        if (n_fail) atomicAdd(&counters->rays_failed, n_fail);
        if (n_ovf) atomicAdd(&counters->stack_overflow, n_ovf);
    }
}

__global__ void k_finalize(RefineArgs a, const int32_t* __restrict__ list, const uint32_t* __restrict__ count,
                           const int32_t* __restrict__ nearest, const int32_t* __restrict__ rep_tri,
                           const uint32_t* __restrict__ dist_bits, const uint32_t* __restrict__ front,
                           const uint32_t* __restrict__ back, float* __restrict__ sdf, rtsdf_counters* counters) {
    const uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li == 0 && counters) atomicAdd(&counters->masked_voxels, count[0]);
    if (li >= count[0]) return;
    const int lin = list[li];
    const float d = __uint_as_float(dist_bits[lin]);
    const uint32_t fr = front[lin], bk = back[lin];
    bool neg = bk > fr;
    if (fr == bk && a.fallback) {
        const int32_t s = nearest[lin];
        const int64_t sl = ((int64_t)((s >> 20) & 1023) * a.g.ny + ((s >> 10) & 1023)) * a.g.nx + (s & 1023);
        float3 A, B, C;
        load_tri(a.verts, a.V, a.tris, rep_tri[sl], a.g, A, B, C);
        const int64_t plane = (int64_t)a.g.nx * a.g.ny;
        const int k = (int)(lin / plane), rem = (int)(lin - (int64_t)k * plane);
        const int j = rem / a.g.nx, i = rem - j * a.g.nx;
        const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
        const float3 n = cross3(sub3(B, A), sub3(C, A));
        neg = dot3(sub3(p, A), n) < 0.0f;
    }
    sdf[lin] = neg ? -d : d;
}

rtsdf_status refine(const rtsdf_grid& gh, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                    const void* bvh, const int32_t* nearest, const int32_t* rep_tri, const rtsdf_refine_params& p,
                    uint32_t* dist_bits, uint32_t* front, uint32_t* back, float* sdf, void* ws,
                    rtsdf_counters* counters, cudaStream_t s) {
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
    RefineWs w;
    refine_ws_layout(gh, static_cast<char*>(ws), &w);
    const int64_t nvox = (int64_t)gh.nx * gh.ny * gh.nz;
    const auto* hdr = static_cast<const BvhHeader*>(bvh);
    const auto* nodes = reinterpret_cast<const BvhNode*>(static_cast<const char*>(bvh) + bvh_nodes_offset());
    const auto* leaves = reinterpret_cast<const BvhLeaf*>(static_cast<const char*>(bvh) + bvh_leaves_offset(T));
    RTSDF_CUDA(cudaMemsetAsync(w.count, 0, 16, s));
    k_resolve<<<(unsigned)((nvox + 255) / 256), 256, 0, s>>>(a, nearest, rep_tri, dist_bits, front, back, sdf, w.list,
                                                            w.count);
    RTSDF_LAUNCHED();
    k_trace<<<num_sms() * 8, 256, 0, s>>>(a, hdr, nodes, leaves, w.list, w.count, dist_bits, front, back, counters);
    RTSDF_LAUNCHED();
    k_finalize<<<(unsigned)((nvox + 255) / 256), 256, 0, s>>>(a, w.list, w.count, nearest, rep_tri, dist_bits, front,
                                                             back, sdf, counters);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
