// 3D jump flooding (Sec. 2.2): one launch per offset k, Jacobi ping-pong.
//
// Candidate comparison: the key of a candidate seed s for voxel v is the integer
// |v - s|^2, ties to the lower packed seed.  The empty marker (-1 = 0xFFFFFFFF)
// decodes to z = 4095, farther than any real seed from every voxel of a grid with
// dims <= 1023, so it loses every comparison against a real seed and needs no
// branch of its own; a candidate equal to the current best is skipped.
#include "rtsdf_device.cuh"
#include "rtsdf_launch.cuh"

namespace rtsdf {

__device__ __forceinline__ int seed_d2(int x, int y, int z, uint32_t s) {
    const int dx = x - (int)(s & 1023u), dy = y - (int)((s >> 10) & 1023u), dz = z - (int)(s >> 20);
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ void consider(int x, int y, int z, uint32_t s, uint32_t& best, int& bd) {
    if (s == best) return;
    const int d = seed_d2(x, y, z, s);
    if (d < bd || (d == bd && s < best)) {
        best = s;
        bd = d;
    }
}

// Plane visiting order: planes grouped by residue mod k (z = r, r+k, r+2k, ...), so
// the three planes a pass reads for one voxel (z-k, z, z+k) are touched by blocks
// that run close together in time and stay in L2.
__device__ __forceinline__ int residue_plane(int bz, int nz, int k) {
    const int nq = nz / k, rem = nz - nq * k;
    int r, q;
    if (bz < rem * (nq + 1)) {
        r = bz / (nq + 1);
        q = bz - r * (nq + 1);
    } else {
        const int b2 = bz - rem * (nq + 1);
        r = rem + b2 / nq;
        q = b2 - (r - rem) * nq;
    }
    return r + q * k;
}

constexpr int kBX = 32, kBY = 8;

__global__ void __launch_bounds__(kBX* kBY) k_jfa_pass(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int nx, int ny, int nz, int k) {
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = residue_plane(blockIdx.z, nz, k);
    if (x >= nx || y >= ny) return;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t lin = (int64_t)z * plane + (int64_t)y * nx + x;
    uint32_t best = __ldg(in + lin);
    int bd = seed_d2(x, y, z, best);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int zz = z + dz * k;
        if (zz < 0 || zz >= nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = y + dy * k;
            if (yy < 0 || yy >= ny) continue;
            const uint32_t* row = in + (int64_t)zz * plane + (int64_t)yy * nx;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = x + dx * k;
                if (xx < 0 || xx >= nx) continue;
                consider(x, y, z, __ldg(row + xx), best, bd);
            }
        }
    }
    out[lin] = best;
}

rtsdf_status jfa(const rtsdf_grid& g, int32_t* a, int32_t* b, const int32_t* steps, int32_t nsteps,
                 int32_t** result, cudaStream_t s) {
    uint32_t* src = reinterpret_cast<uint32_t*>(a);
    uint32_t* dst = reinterpret_cast<uint32_t*>(b);
    const dim3 block(kBX, kBY, 1);
    const dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz);
    for (int i = 0; i < nsteps; ++i) {
        k_jfa_pass<<<grid, block, 0, s>>>(src, dst, g.nx, g.ny, g.nz, steps[i]);
        RTSDF_LAUNCHED();
        uint32_t* t = src; src = dst; dst = t;
    }
    *result = reinterpret_cast<int32_t*>(src);
    return RTSDF_OK;
}

}  // namespace rtsdf
