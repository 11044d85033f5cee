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

constexpr int kJX = 32, kJY = 4;  // block of columns (x, y)
constexpr int kChunk = 32;        // outputs per column and block along z (grids of 16 M voxels and more)
constexpr int kChunkSmall = 16;   // the same for smaller grids, which need more threads to fill the GPU
constexpr int kGroupMaxPlanes = kChunk / 2;  // classes this short are grouped per thread

// One thread per (x, y) column and z-chunk of one residue class mod k: the planes
// z = rz + p*k stream past; each loaded tap is decoded once and offered to the
// (up to) three outputs p-1, p, p+1 that read it, so every output voxel costs
// nine tap loads instead of 27.  Output p is complete once plane p+1 is in.
//
// Power-of-two offsets (offset K known at compile time) take specialised paths:
// columns whose 3x3 tap columns lie inside the grid read the nine taps of a plane
// through three row pointers with immediate offsets; columns near the x/y faces
// read only the tap rows inside the grid (1, 2 or 3, warp-uniform) and clamp a
// missing left/right tap to their own column (jfa_column_band).  Only other
// offsets take the bounds-checked generic path.  The specialised paths fold the
// empty marker into the arithmetic instead of branching on it: 0xFFFFFFFF decodes
// to the seed (1023, 1023, 4095), whose squared distance from any voxel of a grid
// with dimensions <= 1023 exceeds 3070^2 > 3 * 1023^2, more than any real seed's,
// so it never wins against one and is the result (the empty marker) only when
// every tap is empty.  The candidate (d', s) is one signed 64-bit key, d' in the high word,
// so the lexicographic argmin is a 64-bit minimum.
//
// The pass is bound by the integer ALU pipe (compares, selects, shifts and masks
// issue at half rate there), while multiply-adds go to the FMA pipe.  So the seed
// is decoded with two shifts and two multiply-adds by the runtime constants
// m20 = -2^20 and m10 = -2^10 (kernel arguments, so they stay multiply-adds)
// instead of masks, and the squared distance is a chain of multiply-adds.
template <int K>
__device__ __forceinline__ void jfa_column_interior(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                    int nx, int64_t plane, int x, int y, int rz, int nq, int q0,
                                                    int q1, int m20, int m10) {
    const int m2x = -2 * x, m2y = -2 * y;
    const int64_t step = (int64_t)K * plane;
    const long long none = 0x7fffffffffffffffll;
    long long a0 = none, a1 = none, a2 = none;  // outputs p-1, p, p+1
    const uint32_t* r0 = in + (int64_t)(rz + (q0 - 1) * K) * plane + (int64_t)(y - K) * nx + x;
    const uint32_t* r1 = r0 + (int64_t)K * nx;
    const uint32_t* r2 = r1 + (int64_t)K * nx;
    for (int p = q0 - 1; p <= q1; ++p) {
        if (p >= 0 && p < nq) {
            const int z = rz + p * K;
            const int m2z_prev = -2 * (z - K), m2z = -2 * z, m2z_next = -2 * (z + K);
            uint32_t t[9];
            t[0] = __ldg(r0 - K); t[1] = __ldg(r0); t[2] = __ldg(r0 + K);
            t[3] = __ldg(r1 - K); t[4] = __ldg(r1); t[5] = __ldg(r1 + K);
            t[6] = __ldg(r2 - K); t[7] = __ldg(r2); t[8] = __ldg(r2 + K);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const uint32_t s = t[i];
                const uint32_t uz = s >> 20;
                const uint32_t r = uz * (uint32_t)m20 + s;  // s - sz * 2^20 (mod 2^32)
                const uint32_t uy = r >> 10;
                const int sx = (int)(uy * (uint32_t)m10 + r);  // r - sy * 2^10
                const int sy = (int)uy, sz = (int)uz;
                int dxy = sx * m2x;
                dxy = sx * sx + dxy;
                dxy = sy * m2y + dxy;
                dxy = sy * sy + dxy;
                dxy = sz * sz + dxy;
                a0 = min(a0, (long long)(((unsigned long long)(uint32_t)(dxy + m2z_prev * sz) << 32) | s));
                a1 = min(a1, (long long)(((unsigned long long)(uint32_t)(dxy + m2z * sz) << 32) | s));
                a2 = min(a2, (long long)(((unsigned long long)(uint32_t)(dxy + m2z_next * sz) << 32) | s));
            }
        }
        const int done = p - 1;
        if (done >= q0 && done < q1) out[(int64_t)(rz + done * K) * plane + (int64_t)y * nx + x] = (uint32_t)a0;
        a0 = a1;
        a1 = a2;
        a2 = none;
        r0 += step;
        r1 += step;
        r2 += step;
    }
}

// Power-of-two offset, columns near the grid's x/y faces: only the NR tap rows
// dy0 .. dy0+NR-1 lie inside the grid (warp-uniform: they depend on y only), and a
// lane whose left or right tap column is outside loads its own column there
// instead (the same candidate offered twice changes no argmin).  Otherwise as
// jfa_column_interior.
template <int K, int NR>
__device__ __forceinline__ void jfa_column_band(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx,
                                                int64_t plane, int x, int y, int dy0, int rz, int nq, int q0, int q1,
                                                int m20, int m10) {
    const int m2x = -2 * x, m2y = -2 * y;
    const int64_t step = (int64_t)K * plane;
    const int offl = x >= K ? -K : 0, offr = x + K < nx ? K : 0;
    const long long none = 0x7fffffffffffffffll;
    long long a0 = none, a1 = none, a2 = none;  // outputs p-1, p, p+1
    const uint32_t* r[NR];
    r[0] = in + (int64_t)(rz + (q0 - 1) * K) * plane + (int64_t)(y + dy0 * K) * nx + x;
#pragma unroll
    for (int i = 1; i < NR; ++i) r[i] = r[i - 1] + (int64_t)K * nx;
    for (int p = q0 - 1; p <= q1; ++p) {
        if (p >= 0 && p < nq) {
            const int z = rz + p * K;
            const int m2z_prev = -2 * (z - K), m2z = -2 * z, m2z_next = -2 * (z + K);
            uint32_t t[3 * NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                t[3 * i] = __ldg(r[i] + offl);
                t[3 * i + 1] = __ldg(r[i]);
                t[3 * i + 2] = __ldg(r[i] + offr);
            }
#pragma unroll
            for (int i = 0; i < 3 * NR; ++i) {
                const uint32_t s = t[i];
                const uint32_t uz = s >> 20;
                const uint32_t rr = uz * (uint32_t)m20 + s;
                const uint32_t uy = rr >> 10;
                const int sx = (int)(uy * (uint32_t)m10 + rr);
                const int sy = (int)uy, sz = (int)uz;
                int dxy = sx * m2x;
                dxy = sx * sx + dxy;
                dxy = sy * m2y + dxy;
                dxy = sy * sy + dxy;
                dxy = sz * sz + dxy;
                a0 = min(a0, (long long)(((unsigned long long)(uint32_t)(dxy + m2z_prev * sz) << 32) | s));
                a1 = min(a1, (long long)(((unsigned long long)(uint32_t)(dxy + m2z * sz) << 32) | s));
                a2 = min(a2, (long long)(((unsigned long long)(uint32_t)(dxy + m2z_next * sz) << 32) | s));
            }
        }
        const int done = p - 1;
        if (done >= q0 && done < q1) out[(int64_t)(rz + done * K) * plane + (int64_t)y * nx + x] = (uint32_t)a0;
        a0 = a1;
        a1 = a2;
        a2 = none;
#pragma unroll
        for (int i = 0; i < NR; ++i) r[i] += step;
    }
}

// Any column, any offset (the non-power-of-two ones): bounds-checked taps, empty taps skipped.
__device__ __forceinline__ void jfa_column_generic(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                   int nx, int ny, int64_t plane, int k, int x, int y, int rz,
                                                   int nq, int q0, int q1) {
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

#define RTSDF_JFA_CASES(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256)

// One thread: output column (x, y) over a block of z-planes of one residue class mod k.
__device__ __forceinline__ void jfa_column(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx, int ny,
                                           int nz, int k, int nchunk, int chunk, int bx, int by, int bz, int m20,
                                           int m10) {
    const int x = bx * kJX + threadIdx.x;
    const int y = by * kJY + threadIdx.y;
    const int rz = bz / nchunk, ch = bz - rz * nchunk;
    const int nq = (nz - rz + k - 1) / k;  // planes of this residue class
    const int q0 = ch * chunk, q1 = min(nq, q0 + chunk);
    if (x >= nx || y >= ny || q0 >= q1) return;
    const int64_t plane = (int64_t)nx * ny;
    // tap rows inside the grid (warp-uniform) and whether every lane's tap columns are
    const bool ylo = y >= k, yhi = y + k < ny;
    const bool xin = __all_sync(__activemask(), x >= k && x + k < nx);
    switch (k) {
#define RTSDF_JFA_ONE(K)                                                                                          \
    case K:                                                                                                       \
        if (ylo && yhi) {                                                                                         \
            if (xin)                                                                                              \
                jfa_column_interior<K>(in, out, nx, plane, x, y, rz, nq, q0, q1, m20, m10);                       \
            else                                                                                                  \
                jfa_column_band<K, 3>(in, out, nx, plane, x, y, -1, rz, nq, q0, q1, m20, m10);                    \
        } else if (ylo || yhi) {                                                                                  \
            jfa_column_band<K, 2>(in, out, nx, plane, x, y, ylo ? -1 : 0, rz, nq, q0, q1, m20, m10);              \
        } else {                                                                                                  \
            jfa_column_band<K, 1>(in, out, nx, plane, x, y, 0, rz, nq, q0, q1, m20, m10);                         \
        }                                                                                                         \
        return;
        RTSDF_JFA_CASES(RTSDF_JFA_ONE)
#undef RTSDF_JFA_ONE
        default: break;
    }
    jfa_column_generic(in, out, nx, ny, plane, k, x, y, rz, nq, q0, q1);
}

// Large offsets (every residue class holds at most kGroupMaxPlanes planes): one
// thread takes grp consecutive classes of its column, so its fixed costs are spread
// over about kChunk outputs.  Its own kernel, so the loop does not weigh on the
// register allocation of the common path.
template <int K>
__device__ __forceinline__ void jfa_column_grouped_k(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int nx, int ny, int nz, int64_t plane, int x, int y, int rz0,
                                                     int grp, bool xin, int m20, int m10) {
    const bool ylo = y >= K, yhi = y + K < ny;
    for (int c = 0; c < grp; ++c) {
        const int rz = rz0 + c;
        if (rz >= K || rz >= nz) break;
        const int nq = (nz - rz + K - 1) / K;
        if (ylo && yhi) {
            if (xin)
                jfa_column_interior<K>(in, out, nx, plane, x, y, rz, nq, 0, nq, m20, m10);
            else
                jfa_column_band<K, 3>(in, out, nx, plane, x, y, -1, rz, nq, 0, nq, m20, m10);
        } else if (ylo || yhi) {
            jfa_column_band<K, 2>(in, out, nx, plane, x, y, ylo ? -1 : 0, rz, nq, 0, nq, m20, m10);
        } else {
            jfa_column_band<K, 1>(in, out, nx, plane, x, y, 0, rz, nq, 0, nq, m20, m10);
        }
    }
}

template <int K>
__device__ __forceinline__ void jfa_column_grouped(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                   int nx, int ny, int nz, int grp, int bx, int by, int bz, int m20,
                                                   int m10) {
    const int x = bx * kJX + threadIdx.x;
    const int y = by * kJY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const bool xin = __all_sync(__activemask(), x >= K && x + K < nx);
    jfa_column_grouped_k<K>(in, out, nx, ny, nz, (int64_t)nx * ny, x, y, bz * grp, grp, xin, m20, m10);
}

}  // namespace rtsdf
