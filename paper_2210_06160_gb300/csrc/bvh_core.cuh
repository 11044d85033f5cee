// Device parts of the linear BVH build (Morton keys, Karras topology, leaf records
// and bottom-up boxes), shared by the single-scene build (bvh.cu) and the batched
// one (batch.cu).
//
// The boxes only cull ray/triangle tests, so they are padded well beyond FP32
// rounding of the slab test: a triangle that the exact Moller-Trumbore test
// accepts is never culled, and the result of a ray query equals the brute-force
// closest hit over all triangles, whatever the tree looks like.
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

constexpr uint32_t kInvalidKey = 1u << 30;  // after every 30-bit Morton code

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 1023u;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 30-bit Morton code of triangle t's centroid in the grid box, or kInvalidKey for a
// triangle every kernel skips (which then sorts after all valid ones).  Also writes
// the triangle's voxel-space record tv[t].
__device__ __forceinline__ uint32_t tri_morton(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris,
                                               int t, const GridD& g, TriVox* __restrict__ tv) {
    float3 a, b, c;
    const bool ok = load_tri(verts, V, tris, t, g, a, b, c);
    store_tri_vox(tv, t, ok, a, b, c);
    if (!ok) return kInvalidKey;
    const float scale = 1024.0f / (float)max(g.nx, max(g.ny, g.nz));
    const float cx = (a.x + b.x + c.x) * (1.0f / 3.0f), cy = (a.y + b.y + c.y) * (1.0f / 3.0f),
                cz = (a.z + b.z + c.z) * (1.0f / 3.0f);
    const uint32_t qx = (uint32_t)fminf(fmaxf(cx * scale, 0.0f), 1023.0f);
    const uint32_t qy = (uint32_t)fminf(fmaxf(cy * scale, 0.0f), 1023.0f);
    const uint32_t qz = (uint32_t)fminf(fmaxf(cz * scale, 0.0f), 1023.0f);
    return (spread10(qz) << 2) | (spread10(qy) << 1) | spread10(qx);
}

// ------------------------------------------------------------ topology

// Common-prefix length of sorted keys i and j (equal keys: extended by the index
// bits), -1 outside [0, n).
__device__ __forceinline__ int karras_delta(const uint32_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz(i ^ j);
    return __clz(a ^ b);
}
__device__ __forceinline__ int karras_delta(const unsigned long long* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const unsigned long long a = k[i], b = k[j];
    if (a == b) return 64 + __clz(i ^ j);
    return __clzll(a ^ b);
}

// Inner node i of the radix tree over n sorted keys (Karras, HPG 2012): its range,
// split and children; records the children's parents.
template <typename K>
__device__ __forceinline__ void bvh_topology_node(const K* __restrict__ keys, int n, int i, BvhNode* __restrict__ nodes,
                                                  int32_t* __restrict__ parent_inner,
                                                  int32_t* __restrict__ parent_leaf) {
    const int d = (karras_delta(keys, n, i, i + 1) - karras_delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = karras_delta(keys, n, i, i - d);
    int lmax = 2;
    while (karras_delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (karras_delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = karras_delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (karras_delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const bool left_leaf = min(i, j) == gamma, right_leaf = max(i, j) == gamma + 1;
    const int c0 = left_leaf ? ~gamma : gamma, c1 = right_leaf ? ~(gamma + 1) : gamma + 1;
    nodes[i].lo0.w = __int_as_float(c0);
    nodes[i].hi0.w = __int_as_float(c1);
    if (left_leaf) parent_leaf[gamma] = i; else parent_inner[gamma] = i;
    if (right_leaf) parent_leaf[gamma + 1] = i; else parent_inner[gamma + 1] = i;
    if (i == 0) parent_inner[0] = -1;
}

// ------------------------------------------------------------ leaves + boxes

__device__ __forceinline__ float pad_of(float x) { return 0.015625f + fabsf(x) * 3.814697265625e-6f; }

__device__ __forceinline__ void write_slot(BvhNode* node, int slot, float3 lo, float3 hi) {
    float* f = reinterpret_cast<float*>(node) + slot * 8;  // lo at f[0..2], hi at f[4..6]
    __stcg(f + 0, lo.x); __stcg(f + 1, lo.y); __stcg(f + 2, lo.z);
    __stcg(f + 4, hi.x); __stcg(f + 5, hi.y); __stcg(f + 6, hi.z);
}

// Leaf j (triangle tri) of a tree with n leaves: its record, then the boxes of its
// ancestors bottom-up (the second child to arrive at a node continues upward).
__device__ __forceinline__ void bvh_leaf_up(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris,
                                            const GridD& g, int tri, int j, int n, BvhNode* __restrict__ nodes,
                                            BvhLeaf* __restrict__ leaves, const int32_t* __restrict__ parent_inner,
                                            const int32_t* __restrict__ parent_leaf, uint32_t* __restrict__ visits) {
    float3 a, b, c;
    load_tri(verts, V, tris, tri, g, a, b, c);  // valid: invalid keys sort after the n valid ones
    const float3 e1 = sub3(b, a), e2 = sub3(c, a);
    leaves[j].v0 = make_float4(a.x, a.y, a.z, __int_as_float(tri));
    leaves[j].e1 = make_float4(e1.x, e1.y, e1.z, 0.0f);
    leaves[j].e2 = make_float4(e2.x, e2.y, e2.z, 0.0f);
    {
        // centre of the smallest sphere around the triangle: the midpoint of the side
        // opposite an obtuse (or right) angle, else the circumcentre; the radius is then
        // measured to the three vertices, so the sphere holds them whatever the rounding
        const float3 ab = sub3(b, a), ac = sub3(c, a), bc = sub3(c, b);
        const float3 w = cross3(ab, ac);
        const float w2 = dot3(w, w);
        float3 cen;
        if (dot3(ab, ac) <= 0.0f) {
            cen = make_float3(0.5f * (b.x + c.x), 0.5f * (b.y + c.y), 0.5f * (b.z + c.z));
        } else if (-dot3(ab, bc) <= 0.0f) {
            cen = make_float3(0.5f * (a.x + c.x), 0.5f * (a.y + c.y), 0.5f * (a.z + c.z));
        } else if (dot3(ac, bc) <= 0.0f) {
            cen = make_float3(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z));
        } else if (w2 > 0.0f) {
            const float sab = dot3(ab, ab), sac = dot3(ac, ac);
            const float3 p = cross3(ac, w), q = cross3(w, ab);
            const float inv = 0.5f / w2;
            cen = make_float3(a.x + (sab * p.x + sac * q.x) * inv, a.y + (sab * p.y + sac * q.y) * inv,
                              a.z + (sab * p.z + sac * q.z) * inv);
        } else {
            cen = make_float3((a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f),
                              (a.z + b.z + c.z) * (1.0f / 3.0f));
        }
        const float3 da = sub3(a, cen), db = sub3(b, cen), dc = sub3(c, cen);
        const float r = sqrtf(fmaxf(fmaxf(dot3(da, da), dot3(db, db)), dot3(dc, dc)));
        // margin far above the FP32 rounding of any accepted hit point
        const float pad = 0.01f + 1e-5f * (fabsf(cen.x) + fabsf(cen.y) + fabsf(cen.z) + r);
        leaves[j].sph = make_float4(cen.x, cen.y, cen.z, r + pad);
        const float3 n = cross3(e1, e2);
        const float nl = sqrtf(dot3(n, n));
        const float3 nu = nl > 0.0f ? make_float3(n.x / nl, n.y / nl, n.z / nl) : make_float3(0.f, 0.f, 0.f);
        leaves[j].pln = make_float4(nu.x, nu.y, nu.z, dot3(nu, a));
    }
    float3 lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z));
    float3 hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z));
    lo = make_float3(lo.x - pad_of(lo.x), lo.y - pad_of(lo.y), lo.z - pad_of(lo.z));
    hi = make_float3(hi.x + pad_of(hi.x), hi.y + pad_of(hi.y), hi.z + pad_of(hi.z));
    if (n == 1) {  // a single leaf: root with the leaf and a box no ray reaches
        const float far = -3.0e38f;
        nodes[0].lo0 = make_float4(lo.x, lo.y, lo.z, __int_as_float(~0));
        nodes[0].hi0 = make_float4(hi.x, hi.y, hi.z, __int_as_float(~0));
        nodes[0].lo1 = make_float4(far, far, far, 0.0f);
        nodes[0].hi1 = make_float4(far, far, far, 0.0f);
        return;
    }
    int p = parent_leaf[j];
    if (p < 0 || p >= n - 1) return;
    int slot = (__float_as_int(nodes[p].lo0.w) == ~j) ? 0 : 1;
    write_slot(nodes + p, slot, lo, hi);
    __threadfence();
    // a well-formed radix tree over unique 64-bit (code, position) keys is at most
    // 64 levels deep; the bound only protects against a malformed topology
    for (int level = 0; level < 96; ++level) {
        if (p < 0 || p >= n - 1) return;
        if (atomicAdd(visits + p, 1u) == 0) return;  // the sibling's thread continues
        __threadfence();
        const float* f = reinterpret_cast<const float*>(nodes + p);
        const float3 l0 = make_float3(__ldcg(f + 0), __ldcg(f + 1), __ldcg(f + 2));
        const float3 h0 = make_float3(__ldcg(f + 4), __ldcg(f + 5), __ldcg(f + 6));
        const float3 l1 = make_float3(__ldcg(f + 8), __ldcg(f + 9), __ldcg(f + 10));
        const float3 h1 = make_float3(__ldcg(f + 12), __ldcg(f + 13), __ldcg(f + 14));
        lo = make_float3(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z));
        hi = make_float3(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z));
        const int pp = parent_inner[p];
        if (pp < 0 || pp >= n - 1) return;
        slot = (__float_as_int(nodes[pp].lo0.w) == p) ? 0 : 1;
        write_slot(nodes + pp, slot, lo, hi);
        __threadfence();
        p = pp;
    }
}

}  // namespace rtsdf
