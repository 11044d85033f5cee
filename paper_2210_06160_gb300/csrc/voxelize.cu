// Conservative voxelization (Sec. 2.2): seeds and representative triangles.
//
// Work decomposition: every valid triangle covers the bricks (8^3 voxels) of its
// voxel range; a scan over the per-triangle brick counts turns the set of all
// (triangle, brick) pairs into one virtual index space that warps stride over in
// contiguous chunks of 32 items (one binary search per chunk, no pair list, no host
// sync).  Each lane takes one item of the chunk: it tests its triangle against its
// brick (slightly enlarged, so the brick cull never rejects a voxel the voxel test
// accepts), and the voxel tests of the chunk's items on (brick ∩ triangle range)
// are then spread over the lanes (vox_chunk); an overlapping voxel takes the 64-bit
// key (float bits of the closest-point distance^2, triangle id) with atomicMin,
// which is the argmin with ties to the lower id in any order.
#include "rtsdf_launch.cuh"
#include "voxelize_core.cuh"

namespace rtsdf {

constexpr int kChunk = 32;  // items per warp chunk (one per lane)

// Per triangle: number of bricks its voxel range touches (0 if invalid or outside).
__global__ void k_vox_count(const float* __restrict__ verts, int V, const int32_t* __restrict__ tris, int T,
                            GridD g, uint32_t* __restrict__ counts, rtsdf_counters* counters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    float3 a, b, c;
    uint32_t n = 0;
    if (!load_tri(verts, V, tris, t, g, a, b, c)) {
        if (counters) atomicAdd(&counters->skipped_triangles, 1u);
    } else {
        TriRange r;
        if (tri_range(a, b, c, g, r)) n = range_bricks(r);
    }
    counts[t] = n;
}

__global__ void __launch_bounds__(256, 3) k_vox_test(const float* __restrict__ verts, int V,
                                                  const int32_t* __restrict__ tris, int T, GridD g,
                                                  const uint64_t* __restrict__ offsets,  // T+1 exclusive scan
                                                  unsigned long long* __restrict__ keys) {
    const int64_t warp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / kWarp;
    const uint64_t total = offsets[T];
    const uint64_t nchunks = (total + kChunk - 1) / kChunk;
    for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
        const uint64_t i0 = ch * kChunk, i1 = (i0 + kChunk < total) ? i0 + kChunk : total;
        // triangle owning item i0: last t with offsets[t] <= i0
        int lo = 0, hi = T - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i0) lo = mid; else hi = mid - 1;
        }
        vox_chunk<true>(T, offsets, i0, (int)(i1 - i0), lo,
                  [&](int t, float3& a, float3& b, float3& c, TriRange& r, int& tnx, int& tny,
                      unsigned long long*& tk, int& id) {
                      load_tri(verts, V, tris, t, g, a, b, c);  // count > 0 implies valid
                      tri_range(a, b, c, g, r);
                      tnx = g.nx;
                      tny = g.ny;
                      tk = keys;
                      id = t;
                  },
                  g.nx, g.ny, keys);
    }
}

// key -> (packed seed, representative triangle)
__global__ void k_vox_finalize(const uint4* __restrict__ keys, int64_t nvox, GridD g, int32_t* __restrict__ seed,
                               int32_t* __restrict__ rep) {
    const int64_t v2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // pair of voxels
    const int64_t v = 2 * v2;
    if (v >= nvox) return;
    const uint4 kk = __ldcs(keys + v2);  // two 64-bit keys, streamed once
    const int64_t plane = (int64_t)g.nx * g.ny;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int64_t lin = v + e;
        if (lin >= nvox) break;
        const uint32_t lo = e ? kk.z : kk.x, hi = e ? kk.w : kk.y;
        const bool empty = (lo == 0xFFFFFFFFu && hi == 0xFFFFFFFFu);
        const int k = (int)(lin / plane), rem = (int)(lin - (int64_t)k * plane);
        const int j = rem / g.nx, i = rem - j * g.nx;
        seed[lin] = empty ? RTSDF_EMPTY : pack_seed(i, j, k);
        rep[lin] = empty ? -1 : (int32_t)lo;
    }
}

size_t voxelize_workspace(int32_t T, const rtsdf_grid& g) {
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    size_t off = align_up(sizeof(unsigned long long) * (nvox + 1), 256);  // keys (padded to an even count)
    off += align_up(sizeof(uint32_t) * (size_t)T, 256);                    // counts
    off += align_up(sizeof(uint64_t) * ((size_t)T + 1), 256);              // offsets
    off += scan_u32_to_u64_scratch((size_t)T);
    return off;
}

rtsdf_status voxelize(const float* verts, int32_t V, const int32_t* tris, int32_t T, const rtsdf_grid& gh,
                      int32_t* seed, int32_t* rep_tri, void* ws, rtsdf_counters* counters, cudaStream_t s) {
    const GridD g = to_dev(gh);
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
    char* w = static_cast<char*>(ws);
    auto* keys = reinterpret_cast<unsigned long long*>(w);
    w += align_up(sizeof(unsigned long long) * (size_t)(nvox + 1), 256);
    auto* counts = reinterpret_cast<uint32_t*>(w);
    w += align_up(sizeof(uint32_t) * (size_t)T, 256);
    auto* offsets = reinterpret_cast<uint64_t*>(w);
    w += align_up(sizeof(uint64_t) * ((size_t)T + 1), 256);
    void* scan_tmp = w;

    RTSDF_CUDA(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * (size_t)(nvox + 1), s));
    if (T > 0) {
        k_vox_count<<<(T + 255) / 256, 256, 0, s>>>(verts, V, tris, T, g, counts, counters);
        RTSDF_LAUNCHED();
        RTSDF_TRY(scan_u32_to_u64(counts, offsets, (size_t)T, scan_tmp, s));
        k_vox_test<<<num_sms() * 8, 256, 0, s>>>(verts, V, tris, T, g, offsets, keys);
        RTSDF_LAUNCHED();
    }
    const int64_t npairs = (nvox + 1) / 2;
    k_vox_finalize<<<(unsigned)((npairs + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(keys), nvox, g,
                                                                     seed, rep_tri);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
