// Voxel ranges of triangles for the conservative voxelizer (Sec. 2.2), shared by
// the single-scene (voxelize.cu) and batched (batch.cu) kernels.
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

constexpr int kBrick = 8;

// Voxel range of a triangle along one axis: the closed triangle can touch voxel i
// (spanning [i, i+1]) only if min <= i + 1 and max >= i.
__device__ __forceinline__ bool axis_range(float a, float b, float c, int n, int& lo, int& hi) {
    const float mn = fminf(fminf(a, b), c), mx = fmaxf(fmaxf(a, b), c);
    const float l = fmaxf(ceilf(mn) - 1.0f, 0.0f);
    const float h = fminf(floorf(mx), (float)n - 1.0f);
    if (!(l <= h)) return false;
    lo = (int)l;
    hi = (int)h;
    return true;
}

struct TriRange {
    int lo[3], hi[3];
};

__device__ __forceinline__ bool tri_range(float3 a, float3 b, float3 c, const GridD& g, TriRange& r) {
    return axis_range(a.x, b.x, c.x, g.nx, r.lo[0], r.hi[0]) && axis_range(a.y, b.y, c.y, g.ny, r.lo[1], r.hi[1]) &&
           axis_range(a.z, b.z, c.z, g.nz, r.lo[2], r.hi[2]);
}

// Bricks of a triangle's voxel range.
__device__ __forceinline__ uint32_t range_bricks(const TriRange& r) {
    return (uint32_t)((r.hi[0] / kBrick - r.lo[0] / kBrick + 1) * (r.hi[1] / kBrick - r.lo[1] / kBrick + 1) *
                      (r.hi[2] / kBrick - r.lo[2] / kBrick + 1));
}

// Voxel test of one voxel: closed-cube SAT overlap, then the 64-bit key (closest-point
// distance^2 bits, triangle id) lowered with atomicMin.
__device__ __forceinline__ void vox_voxel(float3 a, float3 b, float3 c, int i, int j, int k, int tri_id,
                                          const GridD& g, unsigned long long* __restrict__ keys) {
    const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
    if (!tri_box_overlap(a, b, c, p, 0.5f)) return;
    const float d2 = closest_d2(p, a, b, c);
    const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned long long)(uint32_t)tri_id;
    const int64_t lin = ((int64_t)k * g.ny + j) * g.nx + i;
    atomicMin(keys + lin, key);
}

// Position of the n-th (0-based) set bit of a 16-bit mask holding more than n set bits.
__device__ __forceinline__ int nth_set_bit16(uint32_t x, int n) {
    int pos = 0;
    int c = __popc(x & 0xFFu);
    if (n >= c) { n -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xFu);
    if (n >= c) { n -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (n >= c) { n -= c; x >>= 2; pos += 2; }
    if (n >= (int)(x & 1u)) pos += 1;
    return pos;
}

// The voxel tests of one (triangle, brick) item: a warp culls the brick (enlarged
// by a margin far above FP32 rounding of the voxel test), then its lanes test the
// voxels of brick ∩ range.  When that sub-box is large (a big triangle, typically a
// slanted plane through its whole bounding box), the voxels whose centres lie
// farther from the triangle's plane than the cube's half-extent along the normal
// (a cube that meets the triangle meets its plane) are dropped first, and the
// remaining ones are compacted over the warp, so the full test runs on dense
// lanes.  The margin (0.02 voxel, above the FP32 rounding of the separating-axis
// test, plus the computed normal's angular error times the distance) keeps every
// voxel that test can accept.
__device__ __forceinline__ void vox_item(float3 a, float3 b, float3 c, const TriRange& r, int local, int tri_id,
                                         const GridD& g, unsigned long long* __restrict__ keys) {
    const int lane = (int)lane_id();
    const int nbx = r.hi[0] / kBrick - r.lo[0] / kBrick + 1;
    const int nby = r.hi[1] / kBrick - r.lo[1] / kBrick + 1;
    const int bx = r.lo[0] / kBrick + local % nbx;
    const int by = r.lo[1] / kBrick + (local / nbx) % nby;
    const int bz = r.lo[2] / kBrick + local / (nbx * nby);
    const float3 bc = make_float3((float)(bx * kBrick) + 0.5f * kBrick, (float)(by * kBrick) + 0.5f * kBrick,
                                  (float)(bz * kBrick) + 0.5f * kBrick);
    if (!tri_box_overlap(a, b, c, bc, 0.5f * kBrick + 0.0625f)) return;
    const int x0 = max(r.lo[0], bx * kBrick), x1 = min(r.hi[0], bx * kBrick + kBrick - 1);
    const int y0 = max(r.lo[1], by * kBrick), y1 = min(r.hi[1], by * kBrick + kBrick - 1);
    const int z0 = max(r.lo[2], bz * kBrick), z1 = min(r.hi[2], bz * kBrick + kBrick - 1);
    const int sx = x1 - x0 + 1, sy = y1 - y0 + 1, nsub = sx * sy * (z1 - z0 + 1);
    const float3 e1 = sub3(b, a), e2 = sub3(c, a);
    const float3 nn = cross3(e1, e2);
    const float len2 = dot3(nn, nn);
    // sin^2 of the angle between the edges; the computed unit normal is off the true one by at
    // most about 8u/sin + 8u radians (u = 2^-24), which the margin below scales by the distance
    // from vertex a to the brick's voxels; slivers (sin < 1e-4) skip the filter
    const float sin2 = len2 / (dot3(e1, e1) * dot3(e2, e2));
    if (nsub <= 2 * kWarp || !(sin2 > 1e-8f) || !isfinite(len2)) {
        for (int v = lane; v < nsub; v += kWarp)
            vox_voxel(a, b, c, x0 + v % sx, y0 + (v / sx) % sy, z0 + v / (sx * sy), tri_id, g, keys);
        return;
    }
    const float inv = rsqrtf(len2);
    const float3 nu = make_float3(nn.x * inv, nn.y * inv, nn.z * inv);
    const float3 da = sub3(bc, a);
    const float span = sqrtf(dot3(da, da)) + 7.0f;  // >= |voxel centre - a| over the brick
    const float ang = 0x1p-21f * rsqrtf(sin2) + 0x1p-20f;  // 8u / sin + 16u, with room for the dot product
    const float reach = 0.5f * (fabsf(nu.x) + fabsf(nu.y) + fabsf(nu.z)) + 0.02f + ang * span;
    // slots of the 8^3 brick, x fastest; lane l holds slots l + 32 it (it < 16)
    static_assert(kBrick == 8, "slot layout assumes 8^3 bricks");
    uint32_t m = 0;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
        const int v = lane + kWarp * it;
        const int i = bx * kBrick + (v & 7), j = by * kBrick + ((v >> 3) & 7), k = bz * kBrick + (v >> 6);
        if (i < x0 || i > x1 || j < y0 || j > y1 || k < z0 || k > z1) continue;
        const float dist = nu.x * ((float)i + 0.5f - a.x) + nu.y * ((float)j + 0.5f - a.y) +
                           nu.z * ((float)k + 0.5f - a.z);
        if (fabsf(dist) <= reach) m |= 1u << it;
    }
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
    const int excl = incl - cnt;
    for (int base = 0; base < total; base += kWarp) {
        const int q = base + lane;
        int owner = 0;  // last lane whose exclusive count is <= q
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, owner + step);
            if (e <= q) owner += step;
        }
        const uint32_t mo = __shfl_sync(0xffffffffu, m, owner);
        const int eo = __shfl_sync(0xffffffffu, excl, owner);
        if (q < total) {
            const int v = owner + kWarp * nth_set_bit16(mo, q - eo);
            vox_voxel(a, b, c, bx * kBrick + (v & 7), by * kBrick + ((v >> 3) & 7), bz * kBrick + (v >> 6), tri_id, g,
                      keys);
        }
    }
}

// The items [i0, i0 + n) (n <= 32) of one warp chunk, item i0 in triangle t0, one
// item per lane.  Each lane finds its item's triangle (a search over the chunk's
// triangle offsets), loads it and culls its brick; the surviving small items (and
// slivers) are then packed, their (triangle, voxel) tests spread over the lanes 32
// at a time, so no lane idles on a brick with few voxels in range, and the brick
// culls run side by side instead of one per warp step.  Items with many voxels and
// a well-shaped triangle take vox_item's warp-wide plane filter, one at a time.
// Every (triangle, voxel) pair vox_item would test is tested once, with the same
// separating-axis test and key, so the keys are the same.  fetch(t, a, b, c, r, nx, ny,
// keys, id) loads item triangle t (a valid triangle: it has items) with its voxel
// range, and names the grid, key array and triangle id its keys take (one scene, or
// the triangle's scene in a batch).  vox_item and vox_voxel use only the grid's nx
// and ny (the key index), so those are what the lanes exchange.
// With kOneGrid every triangle takes the grid (nx1, ny1) and the keys keys1, so the
// lanes exchange nothing of them.
template <bool kOneGrid, class Fetch>
__device__ __forceinline__ void vox_chunk(int T, const uint64_t* __restrict__ offsets, uint64_t i0, int n, int t0,
                                          Fetch&& fetch, int nx1 = 0, int ny1 = 0,
                                          unsigned long long* keys1 = nullptr) {
    const int lane = (int)lane_id();
    const uint64_t item = i0 + (uint64_t)lane;
    const bool has = lane < n;
    // triangle of the lane's item: t0 + #{j < 32 : offsets[t0 + j + 1] <= item}, the
    // chunk's triangle end offsets held one per lane
    const uint64_t endl = t0 + lane < T ? offsets[t0 + lane + 1] : ~0ull;
    const uint64_t e31 = __shfl_sync(0xffffffffu, endl, 31);
    int cnt = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint64_t e = __shfl_sync(0xffffffffu, endl, cnt + step - 1);
        if (e <= item) cnt += step;
    }
    if (e31 <= item) cnt = 32;
    int t = t0 + cnt;
    if (has && cnt == 32)
        while (offsets[t + 1] <= item) ++t;  // a chunk spanning more than 32 triangles (empty ones between)
    float3 a = make_float3(0.f, 0.f, 0.f), b = a, c = a;
    TriRange r{};
    int gnx = 1, gny = 1;  // the grid's row and plane sizes (all vox_voxel needs of it)
    unsigned long long* keys = nullptr;
    int id = 0;
    int local = 0;
    bool keep = false, big = false;
    int x0 = 0, y0 = 0, z0 = 0, sx = 1, sy = 1, nsub = 0;
    if (has) {
        fetch(t, a, b, c, r, gnx, gny, keys, id);
        local = (int)(item - offsets[t]);
        const int nbx = r.hi[0] / kBrick - r.lo[0] / kBrick + 1;
        const int nby = r.hi[1] / kBrick - r.lo[1] / kBrick + 1;
        const int bx = r.lo[0] / kBrick + local % nbx;
        const int by = r.lo[1] / kBrick + (local / nbx) % nby;
        const int bz = r.lo[2] / kBrick + local / (nbx * nby);
        const float3 bc = make_float3((float)(bx * kBrick) + 0.5f * kBrick, (float)(by * kBrick) + 0.5f * kBrick,
                                      (float)(bz * kBrick) + 0.5f * kBrick);
        keep = tri_box_overlap(a, b, c, bc, 0.5f * kBrick + 0.0625f);
        x0 = max(r.lo[0], bx * kBrick);
        y0 = max(r.lo[1], by * kBrick);
        z0 = max(r.lo[2], bz * kBrick);
        sx = min(r.hi[0], bx * kBrick + kBrick - 1) - x0 + 1;
        sy = min(r.hi[1], by * kBrick + kBrick - 1) - y0 + 1;
        nsub = sx * sy * (min(r.hi[2], bz * kBrick + kBrick - 1) - z0 + 1);
        if (keep && nsub > 2 * kWarp) {
            const float3 e1 = sub3(b, a), e2 = sub3(c, a);
            const float3 nn = cross3(e1, e2);
            const float len2 = dot3(nn, nn);
            const float sin2 = len2 / (dot3(e1, e1) * dot3(e2, e2));
            big = sin2 > 1e-8f && isfinite(len2);  // the plane-filtered path of vox_item
        }
    }
    // big items: vox_item, the whole warp on one item
    uint32_t bm = __ballot_sync(0xffffffffu, big);
    while (bm) {
        const int src = __ffs(bm) - 1;
        bm &= bm - 1u;
        const float3 ba = make_float3(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src),
                                      __shfl_sync(0xffffffffu, a.z, src));
        const float3 bb = make_float3(__shfl_sync(0xffffffffu, b.x, src), __shfl_sync(0xffffffffu, b.y, src),
                                      __shfl_sync(0xffffffffu, b.z, src));
        const float3 bcv = make_float3(__shfl_sync(0xffffffffu, c.x, src), __shfl_sync(0xffffffffu, c.y, src),
                                       __shfl_sync(0xffffffffu, c.z, src));
        TriRange br;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            br.lo[d] = __shfl_sync(0xffffffffu, r.lo[d], src);
            br.hi[d] = __shfl_sync(0xffffffffu, r.hi[d], src);
        }
        const GridD bg{kOneGrid ? nx1 : __shfl_sync(0xffffffffu, gnx, src),
                       kOneGrid ? ny1 : __shfl_sync(0xffffffffu, gny, src), 1, 0.f, 0.f, 0.f, 1.f};
        unsigned long long* bk = kOneGrid ? keys1
                                          : reinterpret_cast<unsigned long long*>(__shfl_sync(
                                                0xffffffffu, reinterpret_cast<uintptr_t>(keys), src));
        vox_item(ba, bb, bcv, br, __shfl_sync(0xffffffffu, local, src), __shfl_sync(0xffffffffu, id, src), bg, bk);
    }
    // small items and slivers: their voxel tests packed over the lanes
    const int nl = keep && !big ? nsub : 0;
    int incl = nl;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
    const int excl = incl - nl;
    // v / sx and v / sy as (v * ceil(2^16 / s)) >> 16: exact for v < 4096 and s <= 8
    const int rx = (65536 + sx - 1) / sx, ry = (65536 + sy - 1) / sy;
    for (int base = 0; base < total; base += kWarp) {
        const int q = base + lane;
        int owner = 0;  // last lane whose exclusive count is <= q
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, owner + step);
            if (e <= q) owner += step;
        }
        const float3 oa = make_float3(__shfl_sync(0xffffffffu, a.x, owner), __shfl_sync(0xffffffffu, a.y, owner),
                                      __shfl_sync(0xffffffffu, a.z, owner));
        const float3 ob = make_float3(__shfl_sync(0xffffffffu, b.x, owner), __shfl_sync(0xffffffffu, b.y, owner),
                                      __shfl_sync(0xffffffffu, b.z, owner));
        const float3 oc = make_float3(__shfl_sync(0xffffffffu, c.x, owner), __shfl_sync(0xffffffffu, c.y, owner),
                                      __shfl_sync(0xffffffffu, c.z, owner));
        const int ox = __shfl_sync(0xffffffffu, x0, owner), oy = __shfl_sync(0xffffffffu, y0, owner),
                  oz = __shfl_sync(0xffffffffu, z0, owner);
        const int osx = __shfl_sync(0xffffffffu, sx, owner), osy = __shfl_sync(0xffffffffu, sy, owner);
        const int orx = __shfl_sync(0xffffffffu, rx, owner), ory = __shfl_sync(0xffffffffu, ry, owner);
        const int oid = __shfl_sync(0xffffffffu, id, owner), oe = __shfl_sync(0xffffffffu, excl, owner);
        const GridD og{kOneGrid ? nx1 : __shfl_sync(0xffffffffu, gnx, owner),
                       kOneGrid ? ny1 : __shfl_sync(0xffffffffu, gny, owner), 1, 0.f, 0.f, 0.f, 1.f};
        unsigned long long* ok = kOneGrid ? keys1
                                          : reinterpret_cast<unsigned long long*>(__shfl_sync(
                                                0xffffffffu, reinterpret_cast<uintptr_t>(keys), owner));
        if (q < total) {
            const int v = q - oe;
            const int q1 = (v * orx) >> 16, q2 = (q1 * ory) >> 16;
            vox_voxel(oa, ob, oc, ox + v - q1 * osx, oy + q1 - q2 * osy, oz + q2, oid, og, ok);
        }
    }
}

}  // namespace rtsdf
