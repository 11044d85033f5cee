// Linear BVH built on the device: Morton codes -> stable LSD radix sort ->
// Karras (HPG 2012) radix-tree topology -> bottom-up conservative boxes.
//
// The boxes only cull ray/triangle tests, so they are padded well beyond FP32
// rounding of the slab test: a triangle that the exact Moller-Trumbore test in
// refine.cu accepts is never culled, and the result of a ray query equals the
// brute-force closest hit over all triangles.
#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 keys per tile
constexpr uint32_t kInvalidKey = 1u << 30;             // after every 30-bit Morton code

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 1023u;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_bvh_keys(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris, int T, GridD g,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, BvhHeader* hdr,
                           rtsdf_counters* counters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    float3 a, b, c;
    uint32_t key = kInvalidKey;
    if (load_tri(verts, V, tris, t, g, a, b, c)) {
        const float scale = 1024.0f / (float)max(g.nx, max(g.ny, g.nz));
        const float cx = (a.x + b.x + c.x) * (1.0f / 3.0f), cy = (a.y + b.y + c.y) * (1.0f / 3.0f),
                    cz = (a.z + b.z + c.z) * (1.0f / 3.0f);
        const uint32_t qx = (uint32_t)fminf(fmaxf(cx * scale, 0.0f), 1023.0f);
        const uint32_t qy = (uint32_t)fminf(fmaxf(cy * scale, 0.0f), 1023.0f);
        const uint32_t qz = (uint32_t)fminf(fmaxf(cz * scale, 0.0f), 1023.0f);
        key = (spread10(qz) << 2) | (spread10(qy) << 1) | spread10(qx);
        atomicAdd(&hdr->n_leaves, 1);
    } else if (counters) {
        atomicAdd(&counters->skipped_triangles, 1u);
    }
    keys[t] = key;
    vals[t] = (uint32_t)t;
}

// ------------------------------------------------------------ radix sort

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int n, int shift,
                                                            uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int idx = base + r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: element order within a tile is (round, warp, lane).
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin, int n, int shift,
                                                               const uint64_t* __restrict__ offsets, int ntiles,
                                                               uint32_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t run[256];
    __shared__ uint64_t base[256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    run[tid] = 0;
    base[tid] = offsets[tid * ntiles + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int idx = blockIdx.x * kSortTile + r * kSortThreads + tid;
        const bool valid = idx < n;
        const uint32_t key = valid ? kin[idx] : 0u;
        const uint32_t digit = (key >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? digit : 256u + (uint32_t)lane);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[wid][digit] = __popc(peers);
        __syncthreads();
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = s;
            s += c;
        }
        __syncthreads();
        if (valid) {
            const uint64_t pos = base[digit] + run[digit] + wcnt[wid][digit] + rank;
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
        run[tid] += s;
    }
}

// ------------------------------------------------------------ topology

__device__ __forceinline__ int karras_delta(const uint32_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz(i ^ j);
    return __clz(a ^ b);
}

__global__ void k_bvh_topology(const uint32_t* __restrict__ keys, const BvhHeader* __restrict__ hdr,
                               BvhNode* __restrict__ nodes, int32_t* __restrict__ parent_inner,
                               int32_t* __restrict__ parent_leaf) {
    const int n = hdr->n_leaves;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
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

__global__ void k_bvh_leaves(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris, GridD g,
                             const uint32_t* __restrict__ vals, const BvhHeader* __restrict__ hdr,
                             BvhNode* __restrict__ nodes, BvhLeaf* __restrict__ leaves,
                             const int32_t* __restrict__ parent_inner, const int32_t* __restrict__ parent_leaf,
                             uint32_t* __restrict__ visits) {
    const int n = hdr->n_leaves;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int tri = (int)vals[j];
    float3 a, b, c;
    load_tri(verts, V, tris, tri, g, a, b, c);  // valid: invalid keys sort after the n valid ones
    const float3 e1 = sub3(b, a), e2 = sub3(c, a);
    leaves[j].v0 = make_float4(a.x, a.y, a.z, __int_as_float(tri));
    leaves[j].e1 = make_float4(e1.x, e1.y, e1.z, 0.0f);
    leaves[j].e2 = make_float4(e2.x, e2.y, e2.z, 0.0f);
    {
        const float3 cen = make_float3((a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f),
                                       (a.z + b.z + c.z) * (1.0f / 3.0f));
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

// ------------------------------------------------------------ host side

struct BvhWs {
    uint32_t *ka, *va, *kb, *vb, *hist, *visits;
    int32_t *parent_inner, *parent_leaf;
    uint64_t* offsets;
    void* scan_tmp;
};

static size_t bvh_ws_layout(int32_t T, char* base, BvhWs* w) {
    const size_t n = (size_t)(T > 0 ? T : 1);
    const size_t ntiles = (n + kSortTile - 1) / kSortTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes, 256);
        return p;
    };
    char* ka = take(4 * n);
    char* va = take(4 * n);
    char* kb = take(4 * n);
    char* vb = take(4 * n);
    char* hist = take(4 * 256 * ntiles);
    char* offs = take(8 * (256 * ntiles + 1));
    char* pin = take(4 * n);
    char* pl = take(4 * n);
    char* vis = take(4 * n);
    char* scan = take(scan_u32_to_u64_scratch(256 * ntiles));
    if (w) {
        w->ka = (uint32_t*)ka; w->va = (uint32_t*)va; w->kb = (uint32_t*)kb; w->vb = (uint32_t*)vb;
        w->hist = (uint32_t*)hist; w->offsets = (uint64_t*)offs; w->parent_inner = (int32_t*)pin;
        w->parent_leaf = (int32_t*)pl; w->visits = (uint32_t*)vis; w->scan_tmp = scan;
    }
    return off;
}

size_t bvh_bytes(int32_t T) { return bvh_leaves_offset(T) + sizeof(BvhLeaf) * (size_t)(T > 0 ? T : 1); }
size_t bvh_workspace(int32_t T) { return bvh_ws_layout(T, nullptr, nullptr); }

rtsdf_status build_bvh(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid& gh,
                       void* bvh, void* ws, rtsdf_counters* counters, cudaStream_t s) {
    const GridD g = to_dev(gh);
    BvhWs w;
    bvh_ws_layout(T, static_cast<char*>(ws), &w);
    auto* hdr = static_cast<BvhHeader*>(bvh);
    auto* nodes = reinterpret_cast<BvhNode*>(static_cast<char*>(bvh) + bvh_nodes_offset());
    auto* leaves = reinterpret_cast<BvhLeaf*>(static_cast<char*>(bvh) + bvh_leaves_offset(T));
    RTSDF_CUDA(cudaMemsetAsync(hdr, 0, sizeof(BvhHeader), s));
    if (T == 0) return RTSDF_OK;
    k_bvh_keys<<<(T + 255) / 256, 256, 0, s>>>(verts, V, tris, T, g, w.ka, w.va, hdr, counters);
    RTSDF_LAUNCHED();
    const int ntiles = (T + kSortTile - 1) / kSortTile;
    uint32_t *kin = w.ka, *vin = w.va, *kout = w.kb, *vout = w.vb;
    for (int shift = 0; shift < 32; shift += 8) {
        k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(kin, T, shift, w.hist, ntiles);
        RTSDF_LAUNCHED();
        RTSDF_TRY(scan_u32_to_u64(w.hist, w.offsets, (size_t)256 * ntiles, w.scan_tmp, s));
        k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(kin, vin, T, shift, w.offsets, ntiles, kout, vout);
        RTSDF_LAUNCHED();
        uint32_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    // 4 passes: sorted keys/values are back in (ka, va)
    RTSDF_CUDA(cudaMemsetAsync(w.visits, 0, sizeof(uint32_t) * (size_t)T, s));
    k_bvh_topology<<<(T + 255) / 256, 256, 0, s>>>(kin, hdr, nodes, w.parent_inner, w.parent_leaf);
    RTSDF_LAUNCHED();
    k_bvh_leaves<<<(T + 255) / 256, 256, 0, s>>>(verts, V, tris, g, vin, hdr, nodes, leaves, w.parent_inner,
                                                 w.parent_leaf, w.visits);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
