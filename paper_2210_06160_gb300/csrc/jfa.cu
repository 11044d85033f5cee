// 3D jump flooding (Sec. 2.2): one launch per offset k, Jacobi ping-pong.  Offsets
// 64..256 whose residue classes hold at most kGroupMaxPlanes planes run the grouped
// kernel (several classes per thread); the others one class chunk per thread.
#include "jfa_core.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

__global__ void __launch_bounds__(kJX* kJY) k_jfa_pass(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int nx, int ny, int nz, int k, int nchunk, int chunk) {
    jfa_column(in, out, nx, ny, nz, k, nchunk, chunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int K>
__global__ void __launch_bounds__(kJX* kJY) k_jfa_pass_grouped(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out, int nx, int ny, int nz,
                                                             int grp) {
    jfa_column_grouped<K>(in, out, nx, ny, nz, grp, blockIdx.x, blockIdx.y, blockIdx.z);
}

rtsdf_status jfa(const rtsdf_grid& g, int32_t* a, int32_t* b, const int32_t* steps, int32_t nsteps,
                 int32_t** result, cudaStream_t s) {
    uint32_t* src = reinterpret_cast<uint32_t*>(a);
    uint32_t* dst = reinterpret_cast<uint32_t*>(b);
    const dim3 block(kJX, kJY, 1);
    const int chunk = (int64_t)g.nx * g.ny * g.nz >= (int64_t)(16 << 20) ? kChunk : kChunkSmall;
    for (int i = 0; i < nsteps; ++i) {
        const int k = steps[i];
        const int nq = (g.nz + k - 1) / k;
        const int nchunk = (nq + chunk - 1) / chunk;
        const bool pow2 = k >= 64 && k <= 256 && (k & (k - 1)) == 0;
        const unsigned gx = (unsigned)jfa_xblocks(g.nx, k), gy = (unsigned)((g.ny + kJY - 1) / kJY);
        if (pow2 && nq <= kGroupMaxPlanes) {
            const int grp = kGroupOutputs / nq;
            const dim3 grid(gx, gy, (unsigned)((k + grp - 1) / grp));
            if (k == 64)
                k_jfa_pass_grouped<64><<<grid, block, 0, s>>>(src, dst, g.nx, g.ny, g.nz, grp);
            else if (k == 128)
                k_jfa_pass_grouped<128><<<grid, block, 0, s>>>(src, dst, g.nx, g.ny, g.nz, grp);
            else
                k_jfa_pass_grouped<256><<<grid, block, 0, s>>>(src, dst, g.nx, g.ny, g.nz, grp);
        } else {
            const dim3 grid(gx, gy, (unsigned)(k * nchunk));
            k_jfa_pass<<<grid, block, 0, s>>>(src, dst, g.nx, g.ny, g.nz, k, nchunk, chunk);
        }
        RTSDF_LAUNCHED();
        uint32_t* t = src; src = dst; dst = t;
    }
    *result = reinterpret_cast<int32_t*>(src);
    return RTSDF_OK;
}

}  // namespace rtsdf
