// Device-side building blocks of librtsdf: FP32 geometry with a fixed operation
// order (the library is compiled with -fmad=false, so no product is fused into an
// add and every decision below is a pure function of IEEE FP32 operations),
// Philox4x32-10, and the layouts of the internal buffers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rtsdf.h"

namespace rtsdf {

constexpr int kWarp = 32;

// ------------------------------------------------------------------ grid

struct GridD {
    int nx, ny, nz;
    float ox, oy, oz, h;
};

__host__ __device__ inline GridD to_dev(const rtsdf_grid& g) {
    return GridD{g.nx, g.ny, g.nz, g.origin[0], g.origin[1], g.origin[2], g.h};
}

__device__ __forceinline__ int32_t pack_seed(int i, int j, int k) { return (k << 20) | (j << 10) | i; }

// world -> voxel coordinates: (v - o) / h, two correctly rounded operations
__device__ __forceinline__ float3 vox_vertex(const float* __restrict__ verts, int id, const GridD& g) {
    const float* v = verts + 3 * (int64_t)id;
    return make_float3((__ldg(v + 0) - g.ox) / g.h, (__ldg(v + 1) - g.oy) / g.h, (__ldg(v + 2) - g.oz) / g.h);
}

__device__ __forceinline__ bool finite3(float3 a) {
    return isfinite(a.x) && isfinite(a.y) && isfinite(a.z);
}

// Loads triangle t in voxel coordinates; false when an index is out of range or
// a coordinate is not finite (such triangles are skipped by every kernel).
__device__ __forceinline__ bool load_tri(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris,
                                         int t, const GridD& g, float3& a, float3& b, float3& c) {
    int i0 = __ldg(tris + 3 * (int64_t)t), i1 = __ldg(tris + 3 * (int64_t)t + 1), i2 = __ldg(tris + 3 * (int64_t)t + 2);
    if (i0 < 0 || i0 >= V || i1 < 0 || i1 >= V || i2 < 0 || i2 >= V) return false;
    a = vox_vertex(verts, i0, g);
    b = vox_vertex(verts, i1, g);
    c = vox_vertex(verts, i2, g);
    return finite3(a) && finite3(b) && finite3(c);
}

// ------------------------------------------------------------------ vectors

__device__ __forceinline__ float3 sub3(float3 x, float3 y) { return make_float3(x.x - y.x, x.y - y.y, x.z - y.z); }
__device__ __forceinline__ float dot3(float3 x, float3 y) { return x.x * y.x + x.y * y.y + x.z * y.z; }
__device__ __forceinline__ float3 cross3(float3 x, float3 y) {
    return make_float3(x.y * y.z - x.z * y.y, x.z * y.x - x.x * y.z, x.x * y.y - x.y * y.x);
}
__device__ __forceinline__ float comp(float3 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

// ------------------------------------------------- triangle / box overlap

// Separating-axis test of a closed triangle against the closed cube of half-size
// hs centred at cen: box normals, triangle normal, 9 edge x box-normal axes.
// Rejection uses strict comparisons, so touching counts as overlap.
__device__ __forceinline__ bool tri_box_overlap(float3 A, float3 B, float3 C, float3 cen, float hs) {
    const float3 v0 = sub3(A, cen), v1 = sub3(B, cen), v2 = sub3(C, cen);
    {
        float mn = fminf(fminf(v0.x, v1.x), v2.x), mx = fmaxf(fmaxf(v0.x, v1.x), v2.x);
        if (mn > hs || mx < -hs) return false;
        mn = fminf(fminf(v0.y, v1.y), v2.y); mx = fmaxf(fmaxf(v0.y, v1.y), v2.y);
        if (mn > hs || mx < -hs) return false;
        mn = fminf(fminf(v0.z, v1.z), v2.z); mx = fmaxf(fmaxf(v0.z, v1.z), v2.z);
        if (mn > hs || mx < -hs) return false;
    }
    const float3 e0 = sub3(v1, v0), e1 = sub3(v2, v1), e2 = sub3(v0, v2);
    {
        const float3 n = cross3(e0, e1);
        const float d = dot3(n, v0);
        const float r = hs * (fabsf(n.x) + fabsf(n.y) + fabsf(n.z));
        if (d > r || d < -r) return false;
    }
    const float3 E[3] = {e0, e1, e2};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // e x X -> components (y, z) = (e.z, -e.y)
        {
            float ap = E[i].z, aq = -E[i].y;
            float p0 = v0.y * ap + v0.z * aq, p1 = v1.y * ap + v1.z * aq, p2 = v2.y * ap + v2.z * aq;
            float mn = fminf(fminf(p0, p1), p2), mx = fmaxf(fmaxf(p0, p1), p2);
            float r = hs * (fabsf(ap) + fabsf(aq));
            if (mn > r || mx < -r) return false;
        }
        // e x Y -> components (z, x) = (e.x, -e.z)
        {
            float ap = E[i].x, aq = -E[i].z;
            float p0 = v0.z * ap + v0.x * aq, p1 = v1.z * ap + v1.x * aq, p2 = v2.z * ap + v2.x * aq;
            float mn = fminf(fminf(p0, p1), p2), mx = fmaxf(fmaxf(p0, p1), p2);
            float r = hs * (fabsf(ap) + fabsf(aq));
            if (mn > r || mx < -r) return false;
        }
        // e x Z -> components (x, y) = (e.y, -e.x)
        {
            float ap = E[i].y, aq = -E[i].x;
            float p0 = v0.x * ap + v0.y * aq, p1 = v1.x * ap + v1.y * aq, p2 = v2.x * ap + v2.y * aq;
            float mn = fminf(fminf(p0, p1), p2), mx = fmaxf(fmaxf(p0, p1), p2);
            float r = hs * (fabsf(ap) + fabsf(aq));
            if (mn > r || mx < -r) return false;
        }
    }
    return true;
}

// ------------------------------------------------ closest point on triangle

// Squared distance from p to triangle ABC: walk of the vertex, edge and face
// Voronoi regions (Ericson, Real-Time Collision Detection, Sec. 5.1.5) in the
// frame where p is the origin.
__device__ __forceinline__ float closest_d2(float3 p, float3 A, float3 B, float3 C) {
    const float3 a = sub3(A, p), b = sub3(B, p), c = sub3(C, p);
    const float3 ab = sub3(b, a), ac = sub3(c, a);
    const float3 pa = make_float3(-a.x, -a.y, -a.z);
    const float d1 = dot3(ab, pa), d2 = dot3(ac, pa);
    if (d1 <= 0.0f && d2 <= 0.0f) return dot3(a, a);
    const float3 pb = make_float3(-b.x, -b.y, -b.z);
    const float d3 = dot3(ab, pb), d4 = dot3(ac, pb);
    if (d3 >= 0.0f && d4 <= d3) return dot3(b, b);
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        const float s = d1 / (d1 - d3);
        const float3 q = make_float3(a.x + s * ab.x, a.y + s * ab.y, a.z + s * ab.z);
        return dot3(q, q);
    }
    const float3 pc = make_float3(-c.x, -c.y, -c.z);
    const float d5 = dot3(ab, pc), d6 = dot3(ac, pc);
    if (d6 >= 0.0f && d5 <= d6) return dot3(c, c);
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        const float s = d2 / (d2 - d6);
        const float3 q = make_float3(a.x + s * ac.x, a.y + s * ac.y, a.z + s * ac.z);
        return dot3(q, q);
    }
    const float va = d3 * d6 - d5 * d4;
    const float e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
        const float s = e43 / (e43 + e56);
        const float3 bc = sub3(c, b);
        const float3 q = make_float3(b.x + s * bc.x, b.y + s * bc.y, b.z + s * bc.z);
        return dot3(q, q);
    }
    const float inv = 1.0f / (va + vb + vc);
    const float sv = vb * inv, sw = vc * inv;
    const float3 q = make_float3(a.x + ab.x * sv + ac.x * sw, a.y + ab.y * sv + ac.y * sw,
                                 a.z + ab.z * sv + ac.z * sw);
    return dot3(q, q);
}

// ------------------------------------------------------------------ Philox

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications with word swap and key mixing; Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Uniform direction on the sphere (Marsaglia 1972): u, v uniform in [-1, 1) from
// the top 24 bits of two Philox words (exact), accepted when 0 < s = u^2 + v^2 < 1;
// direction (2u sqrt(1-s), 2v sqrt(1-s), 1 - 2s).  Two candidate pairs per Philox
// call, the attempt number in the fourth counter word, at most 32 attempts; att0 is
// the first attempt tried (the ones before it are known to have failed).
__device__ __forceinline__ bool sphere_dir(uint32_t voxel, uint32_t ray, uint32_t scene, uint32_t k0,
                                           uint32_t k1, float3& dir, uint32_t att0 = 0u) {
    for (uint32_t att = att0; att < 32; ++att) {
        const uint4 x = philox4x32_10(make_uint4(voxel, ray, scene, att), k0, k1);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const float u = (float)(w[2 * pr] >> 8) * 0x1p-23f - 1.0f;
            const float v = (float)(w[2 * pr + 1] >> 8) * 0x1p-23f - 1.0f;
            const float s = u * u + v * v;
            if (s > 0.0f && s < 1.0f) {
                const float a = 2.0f * sqrtf(1.0f - s);
                dir = make_float3(u * a, v * a, 1.0f - 2.0f * s);
                return true;
            }
        }
    }
    return false;
}

// The first attempt of sphere_dir (attempt 0: its two candidate pairs in order)
// without branches, the same FP32 operations on the accepted pair.  False when both
// pairs are rejected (about 4.6% of draws); the caller then continues with
// sphere_dir from attempt 1, and dir is (0, 0, 1).
__device__ __forceinline__ bool sphere_dir_first(uint32_t voxel, uint32_t ray, uint32_t scene, uint32_t k0,
                                                 uint32_t k1, float3& dir) {
    const uint4 x = philox4x32_10(make_uint4(voxel, ray, scene, 0u), k0, k1);
    const float u0 = (float)(x.x >> 8) * 0x1p-23f - 1.0f, v0 = (float)(x.y >> 8) * 0x1p-23f - 1.0f;
    const float u1 = (float)(x.z >> 8) * 0x1p-23f - 1.0f, v1 = (float)(x.w >> 8) * 0x1p-23f - 1.0f;
    const float s0 = u0 * u0 + v0 * v0, s1 = u1 * u1 + v1 * v1;
    const bool a0 = s0 > 0.0f && s0 < 1.0f, a1 = s1 > 0.0f && s1 < 1.0f;
    const float u = a0 ? u0 : u1, v = a0 ? v0 : v1, s = a0 ? s0 : (a1 ? s1 : 0.75f);
    const float a = 2.0f * sqrtf(1.0f - s);
    dir = a0 || a1 ? make_float3(u * a, v * a, 1.0f - 2.0f * s) : make_float3(0.f, 0.f, 1.f);
    return a0 || a1;
}

// Moller-Trumbore with precomputed edges e1 = B - A, e2 = C - A.  Hit iff
// 0 < t <= tmax; front iff det > 0 (the ray meets the counter-clockwise side).
__device__ __forceinline__ bool ray_tri(float3 o, float3 d, float3 A, float3 e1, float3 e2, float tmax,
                                        float& t, bool& front, float& margin) {
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    if (det == 0.0f) return false;
    const float inv = 1.0f / det;
    const float3 tv = sub3(o, A);
    const float u = dot3(tv, p) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    const float3 q = cross3(tv, e1);
    const float w = dot3(d, q) * inv;
    const float uw = u + w;
    if (w < 0.0f || uw > 1.0f) return false;
    const float tt = dot3(e2, q) * inv;
    if (!(tt > 0.0f && tt <= tmax)) return false;
    t = tt;
    front = det > 0.0f;
    margin = fminf(fminf(u, w), 1.0f - uw);  // smallest barycentric coordinate of the hit
    return true;
}

__device__ __forceinline__ bool ray_tri(float3 o, float3 d, float3 A, float3 e1, float3 e2, float tmax,
                                        float& t, bool& front) {
    float margin;
    return ray_tri(o, d, A, e1, e2, tmax, t, front, margin);
}

// The same test without early exits, for lanes of a warp that test different items:
// every quantity is the FP32 expression above, evaluated unconditionally, and the
// accept conditions are the negations of the early-exit tests (so a NaN compares
// exactly as it does there), combined at the end; the result is bit-identical.
__device__ __forceinline__ bool ray_tri_flat(float3 o, float3 d, float3 A, float3 e1, float3 e2, float tmax,
                                             float& t, bool& front, float& margin) {
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    const float inv = 1.0f / det;
    const float3 tv = sub3(o, A);
    const float u = dot3(tv, p) * inv;
    const float3 q = cross3(tv, e1);
    const float w = dot3(d, q) * inv;
    const float uw = u + w;
    const float tt = dot3(e2, q) * inv;
    const bool hit = det != 0.0f && !(u < 0.0f || u > 1.0f) && !(w < 0.0f || uw > 1.0f) && tt > 0.0f && tt <= tmax;
    t = tt;
    front = det > 0.0f;
    margin = fminf(fminf(u, w), 1.0f - uw);
    return hit;
}

// ------------------------------------------------------------------ BVH layout

// Buffer: header, then max(n-1,1) inner nodes, then n leaves (n = triangle count).
// Inner node: both child boxes + child references (>= 0 inner node, < 0 leaf ~idx).
struct BvhHeader {
    int32_t n_leaves;  // valid triangles (device-written)
    int32_t n_tris;    // capacity (T)
    int32_t pad[14];
};
struct alignas(16) BvhNode {
    float4 lo0;  // xyz, w = child0 (int bits)
    float4 hi0;  // xyz, w = child1 (int bits)
    float4 lo1;
    float4 hi1;
};
struct alignas(16) BvhLeaf {
    float4 v0;   // xyz = vertex A (voxel space), w = triangle id (int bits)
    float4 e1;   // B - A
    float4 e2;   // C - A
    float4 sph;  // smallest enclosing sphere: centre xyz, w = radius + margin (a superset of the triangle)
    float4 pln;  // unit normal xyz (0 for a degenerate triangle), w = normal . A
};

// Triangle t in voxel coordinates, indexed by triangle id (not in tree order): the
// vertices exactly as load_tri computes them, written once per build so that the
// per-voxel passes (coarse distance, sign fallback) read one 48-byte record instead
// of the index triple, three vertices and nine divisions.  a.w = 1 for a valid
// triangle, 0 for one that every kernel skips.
struct alignas(16) TriVox {
    float4 a, b, c;
};

__host__ __device__ inline size_t bvh_nodes_offset() { return sizeof(BvhHeader); }
__host__ __device__ inline size_t bvh_leaves_offset(int32_t T) {
    return sizeof(BvhHeader) + sizeof(BvhNode) * (size_t)(T > 1 ? T - 1 : 1);
}
__host__ __device__ inline size_t bvh_tris_offset(int32_t T) {
    return bvh_leaves_offset(T) + sizeof(BvhLeaf) * (size_t)(T > 0 ? T : 1);
}

__device__ __forceinline__ void store_tri_vox(TriVox* __restrict__ tv, int t, bool ok, float3 a, float3 b, float3 c) {
    tv[t] = ok ? TriVox{make_float4(a.x, a.y, a.z, 1.0f), make_float4(b.x, b.y, b.z, 0.0f),
                        make_float4(c.x, c.y, c.z, 0.0f)}
               : TriVox{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                        make_float4(0.f, 0.f, 0.f, 0.f)};
}

// Triangle t from the table; false for an id out of [0, T) or an invalid triangle.
__device__ __forceinline__ bool load_tri_vox(const TriVox* __restrict__ tv, int T, int t, float3& a, float3& b,
                                             float3& c) {
    if (t < 0 || t >= T) return false;
    const float4 fa = __ldg(&tv[t].a), fb = __ldg(&tv[t].b), fc = __ldg(&tv[t].c);
    a = make_float3(fa.x, fa.y, fa.z);
    b = make_float3(fb.x, fb.y, fb.z);
    c = make_float3(fc.x, fc.y, fc.z);
    return fa.w != 0.0f;
}

// ------------------------------------------------------------------ misc

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace rtsdf
