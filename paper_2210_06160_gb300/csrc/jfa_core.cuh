// The body of one jump-flooding pass (Sec. 2.2), shared by the single-scene
// launch (jfa.cu) and the batched one (batch.cu).
//
// A pass is integer work: each output takes the argmin over 27 candidate seeds
// of |v - s|^2 (ties to the lower packed seed).  Its cost is instructions, not
// bytes, so the kernel is built to touch each input element once per thread
// column: the dependency of a pass only links voxels congruent mod k, and a
// thread streams one (x, y) column along z through its residue class, offering
// every decoded tap to the three outputs that read it.
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

// Candidate key for output voxel v and seed s: d' = |s|^2 - 2 v.s (= |v - s|^2 - |v|^2,
// the same order for a fixed v; exact in int32 for dims <= 1023), ties to the
// lower packed seed.  The empty marker never takes part.
struct Best {
    int d;
    uint32_t s;
};

__device__ __forceinline__ void offer(Best& b, int d, uint32_t s) {
    if (d < b.d || (d == b.d && s < b.s)) {
        b.d = d;
        b.s = s;
    }
}

constexpr int kJX = 32, kJY = 8;  // block of columns (x, y)
constexpr int kChunk = 16;        // outputs per column and block along z

// One thread per (x, y) column and z-chunk of one residue class mod k: the planes
// z = rz + p*k stream past; each loaded tap is decoded once and offered to the
// (up to) three outputs p-1, p, p+1 that read it, so every output voxel costs
// nine tap loads instead of 27.  Output p is complete once plane p+1 is in.
__device__ __forceinline__ void jfa_column(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx, int ny,
                                           int nz, int k, int nchunk, int bx, int by, int bz) {
    const int x = bx * kJX + threadIdx.x;
    const int y = by * kJY + threadIdx.y;
    const int rz = bz / nchunk, ch = bz - rz * nchunk;
    const int nq = (nz - rz + k - 1) / k;  // planes of this residue class
    const int q0 = ch * kChunk, q1 = min(nq, q0 + kChunk);
    if (x >= nx || y >= ny || q0 >= q1) return;
    const int64_t plane = (int64_t)nx * ny;
    const int m2x = -2 * x, m2y = -2 * y;
    const int xl = x - k, xh = x + k, yl = y - k, yh = y + k;
    const bool okxl = xl >= 0, okxh = xh < nx, okyl = yl >= 0, okyh = yh < ny;
    const Best none{0x7fffffff, 0xffffffffu};
    Best a0 = none, a1 = none, a2 = none;  // outputs p-1, p, p+1
    for (int p = q0 - 1; p <= q1; ++p) {
        if (p >= 0 && p < nq) {
            const int z = rz + p * k;
            const uint32_t* base = in + (int64_t)z * plane;
            const int m2z_prev = -2 * (z - k), m2z = -2 * z, m2z_next = -2 * (z + k);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = y + dy * k;
                if ((dy < 0 && !okyl) || (dy > 0 && !okyh)) continue;
                const uint32_t* row = base + (int64_t)yy * nx;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if ((dx < 0 && !okxl) || (dx > 0 && !okxh)) continue;
                    const uint32_t s = __ldg(row + x + dx * k);
                    if (s == 0xffffffffu) continue;
                    const int sx = (int)(s & 1023u), sy = (int)((s >> 10) & 1023u), sz = (int)(s >> 20);
                    const int dxy = sx * sx + sy * sy + sz * sz + m2x * sx + m2y * sy;
                    offer(a0, dxy + m2z_prev * sz, s);  // plane p is z+k for output p-1
                    offer(a1, dxy + m2z * sz, s);       // z for output p
                    offer(a2, dxy + m2z_next * sz, s);  // z-k for output p+1
                }
            }
        }
        const int done = p - 1;
        if (done >= q0 && done < q1) out[(int64_t)(rz + done * k) * plane + (int64_t)y * nx + x] = a0.s;
        a0 = a1;
        a1 = a2;
        a2 = none;
    }
}

}  // namespace rtsdf
