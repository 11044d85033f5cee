// The body of one jump-flooding pass (Sec. 2.2), shared by the single-scene
// launch (jfa.cu) and the batched one (batch.cu).
//
// A pass is arithmetic, not bytes: each output takes the argmin over 27 candidate
// seeds of |v - s|^2, ties to the lower packed seed.  The dependency of a pass only
// links voxels congruent mod k, so a thread streams one (x, y) column along z through
// its residue class; every tap it loads is decoded once and offered to the three
// outputs that read it (planes z - k, z and z + k of the tap's plane z).
#pragma once

#include "rtsdf_device.cuh"

namespace rtsdf {

constexpr int kJX = 32, kJY = 4;  // block of columns (x, y)
constexpr int kChunk = 64;        // outputs per column and block along z (grids of 16 M voxels and more)
constexpr int kChunkSmall = 16;   // the same for smaller grids, which need more threads to fill the GPU
constexpr int kGroupMaxPlanes = 16;  // classes this short are grouped per thread
constexpr int kGroupOutputs = 32;    // outputs a thread of the grouped passes takes (whole classes)

__host__ __device__ __forceinline__ int jfa_xblocks(int nx, int /*k*/) { return (nx + kJX - 1) / kJX; }

// ------------------------------------------------------------------ generic offsets

// Candidate key for the bounds-checked path: d' = |s|^2 - 2 v.s (= |v - s|^2 - |v|^2,
// the same order for a fixed v; exact in int32 for dims <= 1023), ties to the lower
// packed seed.  The empty marker never takes part.
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

// One output column, any offset (the non-power-of-two ones): bounds-checked taps,
// empty taps skipped.  Planes z = rz + p*k stream past; each loaded tap is offered
// to the three outputs p-1, p, p+1 that read it.
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

// ------------------------------------------------------------------ power-of-two offsets
//
// Distances are computed in FP32 on relative coordinates, where every value is an
// integer below 2^24 and so exact: for a tap in plane z_t, a = sx - x, b = sy - y,
// c = sz - z_t; P = a^2 + b^2 + c^2 is its squared distance to the output of plane
// z_t, and those of planes z_t - k and z_t + k are P + k^2 + 2kc and P + k^2 - 2kc.
// The seed is decoded into those coordinates with float bit tricks:
// (s & 0xFFFFF) | 0x4B000000 is the float 2^23 + 1024 sy + sx, whose quotient by 1024
// rounded down (one FMA in round-down mode) is 2^23 + sy; a byte permutation gives
// 2^23 + (s >> 16), and its quotient by 16 rounded down is 2^23 + sz.  The empty
// marker 0xFFFFFFFF decodes to the seed (1023, 1023, 4095), farther from any voxel of
// a grid with dims <= 1023 than every real seed (3070^2 > 3 * 1022^2), so it wins
// only where every tap is empty.  Pairs of taps run through the paired FP32 units
// (two lanes per instruction).
//
// The argmin of a group of candidates that share an output (the taps of one plane)
// takes two phases, each a tree of unsigned minima (__vimin3_u32; on sm_103a each
// lowers to two 2-input minima, measured): H = the minimum of the distance bits
// (non-negative floats order like their bits), then
// L = the minimum of bits(2 (d - H)) + s, which is s for the candidates at
// distance H and at least 2^30 (above every packed seed, 1022 << 20 | ...) for the
// others; where s is the empty marker the sum wraps to at least 2^30 - 1, still above
// every packed seed.  A group's (H, L) is its lexicographic (distance, seed) minimum;
// the three groups of an output (planes z - k, z, z + k) merge as 64-bit (H, L) keys.

__device__ __forceinline__ uint32_t fbits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// a * b + c on two lanes, rounded toward minus infinity (b and c the same on both)
__device__ __forceinline__ float2 ffma2_rd(float2 a, float b, float c) {
    float rx, ry;
    asm("{ .reg .b64 a, b, c, r; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %4}; mov.b64 c, {%5, %5};\n\t"
        "fma.rm.f32x2 r, a, b, c; mov.b64 {%0, %1}, r; }"
        : "=f"(rx), "=f"(ry)
        : "f"(a.x), "f"(a.y), "f"(b), "f"(c));
    return make_float2(rx, ry);
}

// Two taps: squared distances to the output of their plane (P) and of the planes
// one offset below (lo) and above (hi).
template <int K>
__device__ __forceinline__ void tap_dist2(uint32_t s0, uint32_t s1, float cxy, float cy, float cz, float2& P,
                                          float2& lo, float2& hi) {
    constexpr float kK = (float)K, kK2 = (float)K * (float)K;
    const float2 L = f2(__uint_as_float((s0 & 0xFFFFFu) | 0x4B000000u), __uint_as_float((s1 & 0xFFFFFu) | 0x4B000000u));
    const float2 Z = f2(__uint_as_float(__byte_perm(s0, 0x4B00u, 0x5432u)),
                        __uint_as_float(__byte_perm(s1, 0x4B00u, 0x5432u)));
    const float2 syb = ffma2_rd(L, 0x1p-10f, 0x1p23f - 0x1p13f);  // 2^23 + sy
    const float2 szb = ffma2_rd(Z, 0x1p-4f, 0x1p23f - 0x1p19f);   // 2^23 + sz
    const float2 ay = __fadd2_rn(syb, f2(-cy, -cy));
    const float2 t = __fadd2_rn(L, f2(-cxy, -cxy));  // 1024 ay + ax
    const float2 ax = __ffma2_rn(ay, f2(-1024.0f, -1024.0f), t);
    const float2 az = __fadd2_rn(szb, f2(-cz, -cz));
    P = __ffma2_rn(ax, ax, __ffma2_rn(ay, ay, __fmul2_rn(az, az)));
    const float2 Q = __fadd2_rn(P, f2(kK2, kK2));
    lo = __ffma2_rn(az, f2(2.0f * kK, 2.0f * kK), Q);
    hi = __ffma2_rn(az, f2(-2.0f * kK, -2.0f * kK), Q);
}

template <int N>
__device__ __forceinline__ uint32_t min_tree(const uint32_t (&v)[N]) {
    static_assert(N == 3 || N == 6 || N == 9, "groups hold 3, 6 or 9 candidates");
    if constexpr (N == 3) {
        return __vimin3_u32(v[0], v[1], v[2]);
    } else if constexpr (N == 6) {
        return min(__vimin3_u32(v[0], v[1], v[2]), __vimin3_u32(v[3], v[4], v[5]));
    } else {
        return __vimin3_u32(__vimin3_u32(v[0], v[1], v[2]), __vimin3_u32(v[3], v[4], v[5]),
                            __vimin3_u32(v[6], v[7], v[8]));
    }
}

// Lexicographic (distance, seed) minimum of the N candidates (d, s) as the 64-bit key
// (H, L); d holds them in lane pairs, the last pair possibly half used.
template <int N>
__device__ __forceinline__ unsigned long long group_min(const float2 (&d)[(N + 1) / 2], const uint32_t (&s)[N]) {
    constexpr int NP = (N + 1) / 2;
    uint32_t b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = fbits(i & 1 ? d[i / 2].y : d[i / 2].x);
    const uint32_t H = min_tree<N>(b);
    const float m2H = -2.0f * __uint_as_float(H);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float2 e = __ffma2_rn(d[i], f2(2.0f, 2.0f), f2(m2H, m2H));  // 2 (d - H)
        b[2 * i] = fbits(e.x) + s[2 * i];
        if (2 * i + 1 < N) b[2 * i + 1] = fbits(e.y) + s[2 * i + 1];
    }
    return ((unsigned long long)H << 32) | min_tree<N>(b);
}

__device__ __forceinline__ void merge_min(unsigned long long& acc, unsigned long long k) {
    asm("{ .reg .pred p; setp.lt.u64 p, %1, %0; @p mov.b64 %0, %1; }" : "+l"(acc) : "l"(k));
}

// The NR x 3 taps of one plane: rows from `row`, rstep apart; columns x - K, x,
// x + K at the offsets co[], or at compile-time offsets when INTERIOR.
template <int K, int NR, bool INTERIOR>
__device__ __forceinline__ void jfa_load(const uint32_t* __restrict__ row, int64_t rstep, const int (&co)[3],
                                         uint32_t (&s)[3 * NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) s[3 * r + c] = __ldg(row + r * rstep + (INTERIOR ? (c - 1) * K : co[c]));
}

// One plane of the stream: its taps s give three groups: lo and mid merge into the
// accumulators of outputs p - 1 and p, hi becomes that of output p + 1.  A group
// whose output the thread does not store is skipped (nlo, nmid, nhi false;
// warp-uniform): the grouped passes of the largest offsets use this at the ends of
// their short residue classes; the streaming passes compute every group, as the
// branches cost more there than the halo groups they would skip.
template <int K, int NR>
__device__ __forceinline__ void jfa_plane(const uint32_t (&s)[3 * NR], float cxy, float cy, float cz,
                                          unsigned long long& lo, unsigned long long& mid, unsigned long long& hi,
                                          bool nlo, bool nmid, bool nhi) {
    constexpr int N = 3 * NR, NP = (N + 1) / 2;
    float2 P[NP], dlo[NP], dhi[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
        tap_dist2<K>(s[2 * i], s[2 * i + 1 < N ? 2 * i + 1 : 2 * i], cxy, cy, cz, P[i], dlo[i], dhi[i]);
    if (nlo) merge_min(lo, group_min<N>(dlo, s));
    if (nmid) merge_min(mid, group_min<N>(P, s));
    hi = nhi ? group_min<N>(dhi, s) : ~0ull;
}

// One thread: the outputs (x, y, rz + p K), p in [q0, q1), of one residue class mod
// K; NR tap rows y + (dy0 + r) K lie inside the grid (warp-uniform, a warp holds one
// y).  co[] are the tap column offsets x - K, x, x + K, a missing side replaced by
// the thread's own column (offering a candidate twice changes no argmin); INTERIOR
// warps have every lane's three columns inside the grid and read them at
// compile-time offsets.  Planes pa..pb stream past (with PREFETCH the taps of the
// next plane are loaded while the current one is reduced); the loop is unrolled three
// times so that the tap buffers and the accumulators of outputs p - 1, p, p + 1 rotate
// instead of moving.
template <int K, int NR, bool INTERIOR, bool PREFETCH>
__device__ __forceinline__ void jfa_col(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx,
                                        int64_t plane, int x, const int (&co)[3], int y, int dy0, int rz, int nq,
                                        int q0, int q1) {
    constexpr int N = 3 * NR;
    const float cy = 8388608.0f + (float)y;
    const float cxy = 8388608.0f + (float)x + 1024.0f * (float)y;
    unsigned long long A = ~0ull, B = ~0ull, C = ~0ull;
    const int64_t rstep = (int64_t)K * nx;
    const int64_t zstep = (int64_t)K * plane;
    const int pa = max(q0 - 1, 0), pb = min(q1, nq - 1);  // planes read: pa <= pb
    const uint32_t* row = in + (int64_t)(rz + pa * K) * plane + (int64_t)(y + dy0 * K) * nx + (INTERIOR ? x : 0);
    float cz = 8388608.0f + (float)(rz + pa * K);
    uint32_t* o = out + (int64_t)(rz + (pa - 1) * K) * plane + (int64_t)y * nx + x;  // output p - 1
    uint32_t s[N], t[N], u[N];
    if (PREFETCH) jfa_load<K, NR, INTERIOR>(row, rstep, co, s);
    // plane p with taps cur (the next plane's taps go to nxt); then output p - 1 is
    // complete.  Steps run to pb + 1 so that the last output is stored too.
    auto step = [&](int p, uint32_t(&cur)[N], uint32_t(&nxt)[N], unsigned long long& lo,
                    unsigned long long& mid, unsigned long long& hi) {
        if (PREFETCH) {
            if (p < pb) jfa_load<K, NR, INTERIOR>(row + zstep, rstep, co, nxt);
        } else if (p <= pb) {
            jfa_load<K, NR, INTERIOR>(row, rstep, co, cur);
        }
        if (p <= pb)
            jfa_plane<K, NR>(cur, cxy, cy, cz, lo, mid, hi, PREFETCH || (p > q0 && p <= q1),
                             PREFETCH || (p >= q0 && p < q1), PREFETCH || (p + 1 >= q0 && p + 1 < q1));
        if (p - 1 >= q0 && p - 1 < q1) *o = (uint32_t)lo;
        row += zstep;
        o += zstep;
        cz += (float)K;
    };
    for (int p = pa; p <= pb + 1; p += 3) {  // A/B/C: outputs p-1, p, p+1
        step(p, s, t, A, B, C);
        step(p + 1, t, u, B, C, A);
        step(p + 2, u, s, C, A, B);
    }
}

template <int K, bool PREFETCH>
__device__ __forceinline__ void jfa_col_rows(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx,
                                             int ny, int64_t plane, int x, int y, int rz, int nq, int q0, int q1) {
    const bool ylo = y >= K, yhi = y + K < ny;  // tap rows y - K and y + K inside the grid (warp-uniform)
    const int co[3] = {x >= K ? x - K : x, x, x + K < nx ? x + K : x};
    // every lane of the warp reads its three tap columns inside the grid
    const bool inner = __all_sync(__activemask(), x >= K && x + K < nx);
    if (ylo && yhi) {
        if (inner)
            jfa_col<K, 3, true, PREFETCH>(in, out, nx, plane, x, co, y, -1, rz, nq, q0, q1);
        else
            jfa_col<K, 3, false, PREFETCH>(in, out, nx, plane, x, co, y, -1, rz, nq, q0, q1);
    } else if (ylo || yhi) {
        jfa_col<K, 2, false, PREFETCH>(in, out, nx, plane, x, co, y, ylo ? -1 : 0, rz, nq, q0, q1);
    } else {
        jfa_col<K, 1, false, PREFETCH>(in, out, nx, plane, x, co, y, 0, rz, nq, q0, q1);
    }
}

#define RTSDF_JFA_CASES(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256)

// One thread: output column (x, y) over a chunk of z-planes of one residue class mod k.
__device__ __forceinline__ void jfa_column(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int nx, int ny,
                                           int nz, int k, int nchunk, int chunk, int bx, int by, int bz) {
    const int x = bx * kJX + threadIdx.x;
    const int y = by * kJY + threadIdx.y;
    const int rz = bz / nchunk, ch = bz - rz * nchunk;
    const int nq = (nz - rz + k - 1) / k;  // planes of this residue class
    const int q0 = ch * chunk, q1 = min(nq, q0 + chunk);
    if (x >= nx || y >= ny || q0 >= q1) return;
    const int64_t plane = (int64_t)nx * ny;
    switch (k) {
#define RTSDF_JFA_ONE(K)                                                           \
    case K:                                                                        \
        jfa_col_rows<K, true>(in, out, nx, ny, plane, x, y, rz, nq, q0, q1);       \
        return;
        RTSDF_JFA_CASES(RTSDF_JFA_ONE)
#undef RTSDF_JFA_ONE
        default: break;
    }
    jfa_column_generic(in, out, nx, ny, plane, k, x, y, rz, nq, q0, q1);
}

// Large offsets (every residue class holds at most kGroupMaxPlanes planes): one
// thread takes grp consecutive classes of its column, so its fixed costs are spread
// over about kGroupOutputs outputs.  Its own kernel, so the loop does not weigh on the
// register allocation of the common path.
template <int K>
__device__ __forceinline__ void jfa_column_grouped(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                   int nx, int ny, int nz, int grp, int bx, int by, int bz) {
    const int x = bx * kJX + threadIdx.x;
    const int y = by * kJY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int64_t plane = (int64_t)nx * ny;
    for (int c = 0; c < grp; ++c) {
        const int rz = bz * grp + c;
        if (rz >= K || rz >= nz) break;
        const int nq = (nz - rz + K - 1) / K;
        jfa_col_rows<K, false>(in, out, nx, ny, plane, x, y, rz, nq, 0, nq);  // short classes: no prefetch
    }
}

}  // namespace rtsdf
