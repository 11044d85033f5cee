// Linear BVH built on the device: Morton codes -> stable LSD radix sort ->
// Karras (HPG 2012) radix-tree topology -> bottom-up conservative boxes.
//
// The boxes only cull ray/triangle tests, so they are padded well beyond FP32
// rounding of the slab test: a triangle that the exact Moller-Trumbore test in
// refine.cu accepts is never culled, and the result of a ray query equals the
// brute-force closest hit over all triangles.
#include "bvh_core.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 keys per tile

// ------------------------------------------------------------ radix sort

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K* __restrict__ keys, int n, int shift,
                                                            uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int idx = base + r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: element order within a tile is (round, warp, lane).
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const K* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin, int n, int shift,
                                                               const uint64_t* __restrict__ offsets, int ntiles,
                                                               K* __restrict__ kout, uint32_t* __restrict__ vout) {
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
        const K key = valid ? kin[idx] : K(0);
        const uint32_t digit = (uint32_t)(key >> shift) & 255u;
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


template <typename K>
size_t radix_sort_scratch(int n) {
    const size_t ntiles = ((size_t)(n > 0 ? n : 1) + kSortTile - 1) / kSortTile;
    return align_up(4 * 256 * ntiles, 256) + align_up(8 * (256 * ntiles + 1), 256) +
           scan_u32_to_u64_scratch(256 * ntiles);
}

template <typename K>
rtsdf_status radix_sort_pairs(K* ka, uint32_t* va, K* kb, uint32_t* vb, int n, int key_bits, void* scratch,
                              cudaStream_t s, K** sorted_k, uint32_t** sorted_v) {
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    char* w = static_cast<char*>(scratch);
    auto* hist = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * 256 * (size_t)ntiles, 256);
    auto* offsets = reinterpret_cast<uint64_t*>(w);
    w += align_up(8 * (256 * (size_t)ntiles + 1), 256);
    K *kin = ka, *kout = kb;
    uint32_t *vin = va, *vout = vb;
    for (int shift = 0; n > 0 && shift < key_bits; shift += 8) {
        k_sort_hist<K><<<ntiles, kSortThreads, 0, s>>>(kin, n, shift, hist, ntiles);
        RTSDF_LAUNCHED();
        RTSDF_TRY(scan_u32_to_u64(hist, offsets, (size_t)256 * ntiles, w, s));
        k_sort_scatter<K><<<ntiles, kSortThreads, 0, s>>>(kin, vin, n, shift, offsets, ntiles, kout, vout);
        RTSDF_LAUNCHED();
        K* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    *sorted_k = kin;
    *sorted_v = vin;
    return RTSDF_OK;
}

template size_t radix_sort_scratch<uint32_t>(int);
template size_t radix_sort_scratch<unsigned long long>(int);
template rtsdf_status radix_sort_pairs<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int, int, void*,
                                                 cudaStream_t, uint32_t**, uint32_t**);
template rtsdf_status radix_sort_pairs<unsigned long long>(unsigned long long*, uint32_t*, unsigned long long*,
                                                           uint32_t*, int, int, void*, cudaStream_t,
                                                           unsigned long long**, uint32_t**);

// ------------------------------------------------------------ single-scene kernels

__global__ void k_bvh_keys(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris, int T, GridD g,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, BvhHeader* hdr,
                           TriVox* __restrict__ tv, rtsdf_counters* counters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t key = tri_morton(verts, V, tris, t, g, tv);
    if (key != kInvalidKey)
        atomicAdd(&hdr->n_leaves, 1);
    else if (counters)
        atomicAdd(&counters->skipped_triangles, 1u);
    keys[t] = key;
    vals[t] = (uint32_t)t;
}

__global__ void k_bvh_topology(const uint32_t* __restrict__ keys, const BvhHeader* __restrict__ hdr,
                               BvhNode* __restrict__ nodes, int32_t* __restrict__ parent_inner,
                               int32_t* __restrict__ parent_leaf) {
    const int n = hdr->n_leaves;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    bvh_topology_node(keys, n, i, nodes, parent_inner, parent_leaf);
}

__global__ void k_bvh_leaves(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris, GridD g,
                             const uint32_t* __restrict__ vals, const BvhHeader* __restrict__ hdr,
                             BvhNode* __restrict__ nodes, BvhLeaf* __restrict__ leaves,
                             const int32_t* __restrict__ parent_inner, const int32_t* __restrict__ parent_leaf,
                             uint32_t* __restrict__ visits) {
    const int n = hdr->n_leaves;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    bvh_leaf_up(verts, V, tris, g, (int)vals[j], j, n, nodes, leaves, parent_inner, parent_leaf, visits);
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

size_t bvh_bytes(int32_t T) { return bvh_tris_offset(T) + sizeof(TriVox) * (size_t)(T > 0 ? T : 1); }
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
    auto* tv = reinterpret_cast<TriVox*>(static_cast<char*>(bvh) + bvh_tris_offset(T));
    k_bvh_keys<<<(T + 255) / 256, 256, 0, s>>>(verts, V, tris, T, g, w.ka, w.va, hdr, tv, counters);
    RTSDF_LAUNCHED();
    const int ntiles = (T + kSortTile - 1) / kSortTile;
    uint32_t *kin = w.ka, *vin = w.va, *kout = w.kb, *vout = w.vb;
    for (int shift = 0; shift < 32; shift += 8) {
        k_sort_hist<uint32_t><<<ntiles, kSortThreads, 0, s>>>(kin, T, shift, w.hist, ntiles);
        RTSDF_LAUNCHED();
        RTSDF_TRY(scan_u32_to_u64(w.hist, w.offsets, (size_t)256 * ntiles, w.scan_tmp, s));
        k_sort_scatter<uint32_t><<<ntiles, kSortThreads, 0, s>>>(kin, vin, T, shift, w.offsets, ntiles, kout, vout);
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
