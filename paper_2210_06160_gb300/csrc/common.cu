// Device properties and the device-wide exclusive scan used by the voxelizer.
#include <atomic>

#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

static std::atomic<uint64_t> g_launches{0};

void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 counts per block

// Block-local exclusive scan; block totals to sums[].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in, uint64_t* __restrict__ out,
                                                             size_t n, uint64_t* __restrict__ sums) {
    __shared__ uint64_t warp_tot[kScanThreads / 32];
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const size_t idx = base + i;
        const uint64_t x = idx < n ? in[idx] : 0u;
        v[i] = run;
        run += x;
    }
    // exclusive scan of per-thread totals across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += warp_tot[w];
    const uint64_t tpre = wpre + incl - run;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const size_t idx = base + i;
        if (idx < n) out[idx] = v[i] + tpre;
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = tpre + run;
}

// Exclusive scan of the block totals by one block (sequential chunks per thread).
__global__ void __launch_bounds__(1024) k_scan_sums(uint64_t* __restrict__ sums, int nb, uint64_t* __restrict__ total) {
    __shared__ uint64_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    uint64_t s = 0;
    for (int b = b0; b < b1; ++b) s += sums[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const uint64_t x = part[i];
            part[i] = run;
            run += x;
        }
        *total = run;
    }
    __syncthreads();
    uint64_t run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        const uint64_t x = sums[b];
        sums[b] = run;
        run += x;
    }
}

__global__ void k_scan_add(uint64_t* __restrict__ out, size_t n, const uint64_t* __restrict__ sums) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += sums[idx / kScanTile];
}

size_t scan_u32_to_u64_scratch(size_t n) {
    const size_t nb = (n + kScanTile - 1) / kScanTile;
    return align_up(sizeof(uint64_t) * (nb + 1), 256);
}

rtsdf_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, size_t n, void* scratch, cudaStream_t s) {
    if (n == 0) {
        RTSDF_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
        return RTSDF_OK;
    }
    const size_t nb = (n + kScanTile - 1) / kScanTile;
    auto* sums = static_cast<uint64_t*>(scratch);
    k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    RTSDF_LAUNCHED();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, (int)nb, out + n);
    RTSDF_LAUNCHED();
    if (nb > 1) {
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
        RTSDF_LAUNCHED();
    }
    return RTSDF_OK;
}

}  // namespace rtsdf
