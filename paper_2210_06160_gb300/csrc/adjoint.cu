// Field samples and the adjoint of the field samples and the soft-shadow image
// with respect to the mesh vertices and the light direction.
//
// Differentiable function: every discrete choice of the FP32 forward is held
// fixed -- the flooded seed and its representative triangle, the ray mask, the
// front/back vote, the source that set each refined distance (the coarse closest
// point, or the winning ray's hit triangle, recorded by rtsdf_refine_tracked), and
// the raymarch's control flow (stop step, step caps, the sample attaining the
// penumbra minimum, the trilinear cell of each sample, the clamp of the output).
// With those fixed, the field and the two outputs are smooth in the vertices and
// the light, and the adjoint is:
//   closest point (Sec. 2.2, coarse field): d|q - p| / dX_m = lambda_m (q - p) / |q - p|
//       (envelope theorem: q moves within the triangle's plane to first order);
//   ray hit (Sec. 2.1, refined field): t = ((X_0 - p) . n) / (d . n), dt / dX_m = lambda_m n / (d . n)
//       (implicit differentiation of the hit point staying in the triangle's plane);
//   trilinear samples: the corner weights and the interpolant's gradient;
//   raymarch (Sec. 2.4, 2.5.2): reverse mode through t_{s+1} = t_s + min(d_s, cap),
//       d_s = field(o + t_s L) - bias and the penumbra estimate k e / (t - y) at the
//       argmin step, replayed from checkpoints of t every kSeg steps.
// The gradient is accumulated in FP32 with atomics (sum order is not fixed).
#include "rtsdf_launch.cuh"
#include "shadow_march.cuh"

namespace rtsdf {

constexpr int kSeg = 8;                    // raymarch steps between checkpoints
constexpr int kMaxCk = RTSDF_BACKWARD_MAX_STEPS / kSeg;
static_assert(RTSDF_BACKWARD_MAX_STEPS % kSeg == 0, "checkpoint segments must tile the step limit");

struct BwdWs {
    double* gl;   // dLoss / dL for the unit light direction, 3 doubles
    float* gsdf;  // dLoss / d(field), one float per voxel
};

static size_t bwd_layout(const rtsdf_grid& g, char* base, BwdWs* w) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    if (w) {
        w->gl = reinterpret_cast<double*>(base);
        w->gsdf = reinterpret_cast<float*>(base + 256);
    }
    return 256 + align_up(4 * n, 256);
}

size_t backward_workspace(const rtsdf_grid& g) { return bwd_layout(g, nullptr, nullptr); }

// ------------------------------------------------------------------ samples

__device__ __forceinline__ float3 world_to_voxel(const GridD& g, const float* __restrict__ p) {
    return make_float3((__ldg(p) - g.ox) / g.h, (__ldg(p + 1) - g.oy) / g.h, (__ldg(p + 2) - g.oz) / g.h);
}

__global__ void __launch_bounds__(256) k_sample(GridD g, const float* __restrict__ sdf, const float* __restrict__ pts,
                                                int M, float* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const float3 q = world_to_voxel(g, pts + 3 * (int64_t)m);
    out[m] = trilinear(sdf, g, q.x, q.y, q.z);
}

// Corner weights of a cell: products of (1 - f) / f per axis, x fastest.
__device__ __forceinline__ void cell_weights(const Cell& c, float w[8]) {
    const float wx[2] = {1.0f - c.fx, c.fx}, wy[2] = {1.0f - c.fy, c.fy}, wz[2] = {1.0f - c.fz, c.fz};
#pragma unroll
    for (int b = 0; b < 8; ++b) w[b] = wx[b & 1] * wy[(b >> 1) & 1] * wz[b >> 2];
}

// Gradient of the trilinear interpolant with respect to the sample position
// (voxel units).  Along a clamped axis both corners are the same voxel, so the
// differences below vanish there.
__device__ __forceinline__ float3 cell_grad(const float v[8], const Cell& c) {
    const float uy = 1.0f - c.fy, uz = 1.0f - c.fz;
    const float c00 = lerpf(v[0], v[1], c.fx), c10 = lerpf(v[2], v[3], c.fx);
    const float c01 = lerpf(v[4], v[5], c.fx), c11 = lerpf(v[6], v[7], c.fx);
    const float gz = lerpf(c01, c11, c.fy) - lerpf(c00, c10, c.fy);
    const float gy = uz * (c10 - c00) + c.fz * (c11 - c01);
    const float gx = uz * (uy * (v[1] - v[0]) + c.fy * (v[3] - v[2])) + c.fz * (uy * (v[5] - v[4]) + c.fy * (v[7] - v[6]));
    return make_float3(gx, gy, gz);
}

__device__ __forceinline__ void scatter_cell(float* __restrict__ gsdf, const Cell& c, float g) {
    float w[8];
    cell_weights(c, w);
#pragma unroll
    for (int b = 0; b < 8; ++b) atomicAdd(gsdf + c.c[b], g * w[b]);
}

__global__ void __launch_bounds__(256) k_sample_adjoint(GridD g, const float* __restrict__ pts, int M,
                                                        const float* __restrict__ d_samples,
                                                        float* __restrict__ gsdf) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const float gs = __ldg(d_samples + m);
    if (gs == 0.0f) return;
    const float3 q = world_to_voxel(g, pts + 3 * (int64_t)m);
    scatter_cell(gsdf, cell_at(g, q.x, q.y, q.z), gs);
}

// ------------------------------------------------------------------ shadow

// Adjoint of one receiver's visibility, upstream gradient gv.  Replays the march of
// k_shadow with its FP32 samples and steps (so every stop and step decision is the
// forward's) and the penumbra estimate in the quotient form the oracle uses, whose
// first minimum is the sample the frozen function differentiates; then walks the
// steps up to that argmin backwards one checkpoint segment at a time.
// Adds dLoss/d(field) into gsdf and returns dLoss/dL (unit light direction).
__device__ float3 shadow_pixel_adjoint(const ShadowArgs& a, const float* __restrict__ sdf, float3 o, float t0, float gv,
                                       float* __restrict__ gsdf) {
    float ck[kMaxCk];
    float t = t0, res = 1.0f, d_prev = __int_as_float(0x7f800000);
    int argmin = -1;
    bool hit = false, am_tiny = false;
    float am_t = 0.0f, am_d = 0.0f, am_dp = 0.0f, am_y = 0.0f, am_e = 0.0f;
    for (int s = 0; s < a.steps; ++s) {
        if ((s % kSeg) == 0) ck[s / kSeg] = t;
        const float qx = o.x + t * a.L.x, qy = o.y + t * a.L.y, qz = o.z + t * a.L.z;
        if (outside_box(a.g, qx, qy, qz)) break;
        const float d = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
        if (d <= a.hit_eps) {
            hit = true;
            break;
        }
        const float dd = d * d;
        const float y = dd / (2.0f * d_prev);
        const float e = sqrtf(fmaxf(dd - y * y, 0.0f));
        const float r = (a.k * e) / fmaxf(t - y, 1e-6f);
        if (r < res) {  // the running minimum: the first step attaining it
            res = r;
            argmin = s;
            am_t = t;
            am_d = d;
            am_dp = d_prev;
            am_y = y;
            am_e = e;
            am_tiny = !(t - y > 1e-6f);
        }
        d_prev = d;
        t = t + fminf(d, a.max_step);
    }
    float3 gL = make_float3(0.0f, 0.0f, 0.0f);
    // the clamped output is constant on the frozen path
    if (hit || argmin < 0 || !(res > 0.0f) || !(res < 1.0f)) return gL;

    // vis = k e / den at the argmin step i, e = sqrt(d_i^2 - y^2), y = d_i^2 / (2 d_{i-1}),
    // den = t_i - y (or the 1e-6 floor)
    const float den = am_tiny ? 1e-6f : am_t - am_y;
    const float ge = gv * a.k / den;
    float gy = 0.0f, gti = 0.0f, gdi = 0.0f, gdp = 0.0f;
    if (!am_tiny) {
        const float q = gv * a.k * am_e / (den * den);
        gti = -q;
        gy = q;
    }
    if (am_e > 0.0f) {
        gdi = ge * am_d / am_e;
        gy = gy - ge * am_y / am_e;
    }
    if (argmin > 0) {
        gdi = gdi + gy * am_d / am_dp;
        gdp = -gy * am_d * am_d / (2.0f * am_dp * am_dp);
    }

    float gt_next = 0.0f;  // dLoss / dt_{s+1}
    for (int seg = argmin / kSeg; seg >= 0; --seg) {
        const int s0 = seg * kSeg;
        const int n = min(kSeg, argmin - s0 + 1);
        float ts[kSeg], ds[kSeg];
        float tt = ck[seg];
#pragma unroll
        for (int j = 0; j < kSeg; ++j) {
            if (j < n) {
                ts[j] = tt;
                const float qx = o.x + tt * a.L.x, qy = o.y + tt * a.L.y, qz = o.z + tt * a.L.z;
                const float dj = trilinear(sdf, a.g, qx, qy, qz) - a.bias;
                ds[j] = dj;
                tt = tt + fminf(dj, a.max_step);
            }
        }
#pragma unroll
        for (int j = kSeg - 1; j >= 0; --j) {
            if (j < n) {
                const int s = s0 + j;
                float gt, gd;
                if (s == argmin) {
                    gt = gti;
                    gd = gdi;
                } else {
                    gt = gt_next;                                      // t_{s+1} = t_s + ...
                    gd = ds[j] < a.max_step ? gt_next : 0.0f;          // ... + d_s when not capped
                    if (s == argmin - 1) gd = gd + gdp;
                }
                if (gd != 0.0f) {
                    const float qx = o.x + ts[j] * a.L.x, qy = o.y + ts[j] * a.L.y, qz = o.z + ts[j] * a.L.z;
                    const Cell c = cell_at(a.g, qx, qy, qz);
                    float v[8];
                    cell_load(sdf, c, v);
                    scatter_cell(gsdf, c, gd);
                    const float3 gr = cell_grad(v, c);
                    const float3 gq = make_float3(gd * gr.x, gd * gr.y, gd * gr.z);
                    gt = gt + dot3(gq, a.L);
                    gL = make_float3(gL.x + gq.x * ts[j], gL.y + gq.y * ts[j], gL.z + gq.z * ts[j]);
                }
                gt_next = gt;
            }
        }
    }
    return gL;
}

__global__ void __launch_bounds__(128) k_shadow_adjoint(ShadowArgs a_in, const float* __restrict__ sdf,
                                                        const float* __restrict__ pos, const float* __restrict__ nrm,
                                                        int P, const float* __restrict__ d_vis,
                                                        float* __restrict__ gsdf, double* __restrict__ gl) {
    const ShadowArgs a = with_light(a_in);
    __shared__ float red[3][4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float3 g = make_float3(0.0f, 0.0f, 0.0f);
    if (i < P) {
        const float gv = __ldg(d_vis + i);
        if (gv != 0.0f) g = shadow_pixel_adjoint(a, sdf, march_origin(a, pos, nrm, i), march_start(a, i), gv, gsdf);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        g.x += __shfl_xor_sync(0xffffffffu, g.x, off);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, off);
        g.z += __shfl_xor_sync(0xffffffffu, g.z, off);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][warp] = g.x;
        red[1][warp] = g.y;
        red[2][warp] = g.z;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const float s = red[threadIdx.x][0] + red[threadIdx.x][1] + red[threadIdx.x][2] + red[threadIdx.x][3];
        if (s != 0.0f) atomicAdd(gl + threadIdx.x, (double)s);
    }
}

// dLoss/dl for the unnormalised light direction l = |l| L:
// (gL - L (L . gL)) / |l|.
__global__ void k_light_finalize(const double* __restrict__ gl, float3 L, float len, const float* __restrict__ Ldev,
                                 float* __restrict__ d_light) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (Ldev) L = unit_light(Ldev, len);  // the caller's device light vector
    const double lx = L.x, ly = L.y, lz = L.z;
    const double LgL = lx * gl[0] + ly * gl[1] + lz * gl[2];
    d_light[0] = (float)((gl[0] - lx * LgL) / (double)len);
    d_light[1] = (float)((gl[1] - ly * LgL) / (double)len);
    d_light[2] = (float)((gl[2] - lz * LgL) / (double)len);
}

// ------------------------------------------------------------------ field

struct FieldArgs {
    GridD g;
    const float* verts;
    int V;
    const int32_t* tris;
    int T;
    float mask2, inv_h;
    uint32_t k0, k1, scene;
    int fallback;
};

// Closest point of triangle ABC to p, in the frame where p is the origin (the
// Voronoi-region walk of Ericson, Real-Time Collision Detection, Sec. 5.1.5):
// returns q - p and the barycentric weights of q.
__device__ __forceinline__ float3 closest_point_bary(float3 p, float3 A, float3 B, float3 C, float lam[3]) {
    const float3 a = sub3(A, p), b = sub3(B, p), c = sub3(C, p);
    const float3 ab = sub3(b, a), ac = sub3(c, a);
    const float3 pa = make_float3(-a.x, -a.y, -a.z);
    const float d1 = dot3(ab, pa), d2 = dot3(ac, pa);
    if (d1 <= 0.0f && d2 <= 0.0f) {
        lam[0] = 1.0f; lam[1] = 0.0f; lam[2] = 0.0f;
        return a;
    }
    const float3 pb = make_float3(-b.x, -b.y, -b.z);
    const float d3 = dot3(ab, pb), d4 = dot3(ac, pb);
    if (d3 >= 0.0f && d4 <= d3) {
        lam[0] = 0.0f; lam[1] = 1.0f; lam[2] = 0.0f;
        return b;
    }
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        const float s = d1 / (d1 - d3);
        lam[0] = 1.0f - s; lam[1] = s; lam[2] = 0.0f;
        return make_float3(a.x + s * ab.x, a.y + s * ab.y, a.z + s * ab.z);
    }
    const float3 pc = make_float3(-c.x, -c.y, -c.z);
    const float d5 = dot3(ab, pc), d6 = dot3(ac, pc);
    if (d6 >= 0.0f && d5 <= d6) {
        lam[0] = 0.0f; lam[1] = 0.0f; lam[2] = 1.0f;
        return c;
    }
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        const float s = d2 / (d2 - d6);
        lam[0] = 1.0f - s; lam[1] = 0.0f; lam[2] = s;
        return make_float3(a.x + s * ac.x, a.y + s * ac.y, a.z + s * ac.z);
    }
    const float va = d3 * d6 - d5 * d4;
    const float e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
        const float s = e43 / (e43 + e56);
        const float3 bc = sub3(c, b);
        lam[0] = 0.0f; lam[1] = 1.0f - s; lam[2] = s;
        return make_float3(b.x + s * bc.x, b.y + s * bc.y, b.z + s * bc.z);
    }
    const float inv = 1.0f / (va + vb + vc);
    const float sv = vb * inv, sw = vc * inv;
    lam[0] = 1.0f - sv - sw; lam[1] = sv; lam[2] = sw;
    return make_float3(a.x + ab.x * sv + ac.x * sw, a.y + ab.y * sv + ac.y * sw, a.z + ab.z * sv + ac.z * sw);
}

// Per-voxel contribution to the vertex gradient: triangle `tri` gets, at vertex m,
// scale * lam[m] * dir (9 values, m-major).
struct VoxGrad {
    int32_t tri;  // -1: none
    float v[9];
};

__device__ __forceinline__ void set_grad(VoxGrad& o, int tri, const float lam[3], float3 dir, float scale) {
    o.tri = tri;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float s = scale * lam[m];
        o.v[3 * m + 0] = s * dir.x;
        o.v[3 * m + 1] = s * dir.y;
        o.v[3 * m + 2] = s * dir.z;
    }
}

// The frozen source of voxel lin and gsdf(v) * d field(v) / d vertices (world units).
__device__ __forceinline__ VoxGrad voxel_grad(const FieldArgs& a, int64_t lin, const int32_t* __restrict__ nearest,
                                              const int32_t* __restrict__ rep_tri,
                                              const uint32_t* __restrict__ front, const uint32_t* __restrict__ back,
                                              const uint32_t* __restrict__ win_ray,
                                              const int32_t* __restrict__ win_tri, const float* __restrict__ gsdf) {
    VoxGrad o;
    o.tri = -1;
    const GridD& g = a.g;
    const float gs = __ldg(gsdf + lin);
    if (gs == 0.0f) return o;
    const int32_t sd = __ldg(nearest + lin);
    if (sd == RTSDF_EMPTY) return o;  // constant field value
    const int si = sd & 1023, sj = (sd >> 10) & 1023, sk = (sd >> 20) & 1023;
    const int32_t rep = __ldg(rep_tri + ((int64_t)sk * g.ny + sj) * g.nx + si);
    float3 A, B, C;
    if (rep < 0 || rep >= a.T || !load_tri(a.verts, a.V, a.tris, rep, g, A, B, C)) return o;
    const int i = (int)(lin % g.nx), j = (int)((lin / g.nx) % g.ny), k = (int)(lin / ((int64_t)g.nx * g.ny));
    const float3 p = make_float3((float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f);
    const int dx = i - si, dy = j - sj, dz = k - sk;
    const bool masked = (float)(dx * dx + dy * dy + dz * dz) <= a.mask2;
    float sg = 1.0f;
    if (masked) {
        const uint32_t fr = __ldg(front + lin), bk = __ldg(back + lin);
        bool neg = bk > fr;
        if (fr == bk && a.fallback) neg = dot3(sub3(p, A), cross3(sub3(B, A), sub3(C, A))) < 0.0f;
        sg = neg ? -1.0f : 1.0f;
    }
    const uint32_t wr = masked ? __ldg(win_ray + lin) : 0xFFFFFFFFu;
    float lam[3];
    if (wr == 0xFFFFFFFFu) {
        // coarse source: |q - p| (minus beta when unmasked, times the vote when masked)
        const float3 qp = closest_point_bary(p, A, B, C, lam);
        const float u = sqrtf(dot3(qp, qp));
        if (!(u > 0.0f)) return o;
        set_grad(o, rep, lam, qp, gs * sg * a.inv_h / u);
        return o;
    }
    // refined source: the winning ray's hit on its triangle
    const int32_t tri = __ldg(win_tri + lin);
    float3 d;
    if (tri < 0 || tri >= a.T || !sphere_dir((uint32_t)lin, wr, a.scene, a.k0, a.k1, d)) return o;
    if (!load_tri(a.verts, a.V, a.tris, tri, g, A, B, C)) return o;
    const float3 e1 = sub3(B, A), e2 = sub3(C, A), nn = cross3(e1, e2);
    const float3 x0 = sub3(A, p);
    const float dn = dot3(d, nn);
    if (dn == 0.0f) return o;
    const float t = dot3(x0, nn) / dn;
    const float3 ap = make_float3(t * d.x - x0.x, t * d.y - x0.y, t * d.z - x0.z);
    const float n2 = dot3(nn, nn);
    lam[1] = dot3(cross3(ap, e2), nn) / n2;
    lam[2] = dot3(cross3(e1, ap), nn) / n2;
    lam[0] = 1.0f - lam[1] - lam[2];
    set_grad(o, tri, lam, nn, gs * sg * a.inv_h / dn);
    return o;
}

// One thread per voxel (block-strided, warp-uniform trip count): the voxel's
// contribution, then a segmented warp reduction over runs of consecutive lanes with
// the same triangle (neighbouring voxels mostly share their source triangle), and
// one set of atomics per run instead of one per voxel.
__global__ void __launch_bounds__(256) k_field_adjoint(FieldArgs a, const int32_t* __restrict__ nearest,
                                                       const int32_t* __restrict__ rep_tri,
                                                       const uint32_t* __restrict__ front,
                                                       const uint32_t* __restrict__ back,
                                                       const uint32_t* __restrict__ win_ray,
                                                       const int32_t* __restrict__ win_tri,
                                                       const float* __restrict__ gsdf, float* __restrict__ d_verts) {
    const GridD& g = a.g;
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lin = base + threadIdx.x;
        VoxGrad o;
        o.tri = -1;
        if (lin < n) o = voxel_grad(a, lin, nearest, rep_tri, front, back, win_ray, win_tri, gsdf);
        if (o.tri < 0) {
#pragma unroll
            for (int c = 0; c < 9; ++c) o.v[c] = 0.0f;
        }
        if (!__any_sync(0xffffffffu, o.tri >= 0)) continue;
        // runs of equal triangle ids: heads, and the last lane of this lane's run
        const int prev = __shfl_up_sync(0xffffffffu, o.tri, 1);
        const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != o.tri);
        const uint32_t later = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
        const int run_end = later ? __ffs(later) - 2 : 31;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const float u = __shfl_down_sync(0xffffffffu, o.v[c], off);
                if (lane + off <= run_end) o.v[c] += u;
            }
        }
        if (o.tri >= 0 && ((heads >> lane) & 1u)) {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int vid = __ldg(a.tris + 3 * (int64_t)o.tri + m);
                atomicAdd(d_verts + 3 * (int64_t)vid + 0, o.v[3 * m + 0]);
                atomicAdd(d_verts + 3 * (int64_t)vid + 1, o.v[3 * m + 1]);
                atomicAdd(d_verts + 3 * (int64_t)vid + 2, o.v[3 * m + 2]);
            }
        }
    }
}

// ------------------------------------------------------------------ entry points

rtsdf_status sample(const rtsdf_grid& gh, const float* sdf, const float* pts, int32_t M, float* out, cudaStream_t s) {
    if (M == 0) return RTSDF_OK;
    k_sample<<<(M + 255) / 256, 256, 0, s>>>(to_dev(gh), sdf, pts, M, out);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

rtsdf_status backward(const rtsdf_grid& gh, const float* verts, int32_t V, const int32_t* tris, int32_t T,
                      const int32_t* nearest, const int32_t* rep_tri, const uint32_t* front, const uint32_t* back,
                      const uint32_t* win_ray, const int32_t* win_tri, const rtsdf_refine_params& rp,
                      const float* sdf, const float* pts, int32_t M, const float* d_samples, const float* pos,
                      const float* nrm, int32_t P, const rtsdf_shadow_params& sp, const float* d_vis,
                      float* d_verts, float* d_light, void* ws, cudaStream_t s) {
    BwdWs w;
    bwd_layout(gh, static_cast<char*>(ws), &w);
    const size_t nvox = (size_t)gh.nx * gh.ny * gh.nz;
    RTSDF_CUDA(cudaMemsetAsync(w.gl, 0, 3 * sizeof(double), s));
    RTSDF_CUDA(cudaMemsetAsync(w.gsdf, 0, 4 * nvox, s));
    if (V > 0) RTSDF_CUDA(cudaMemsetAsync(d_verts, 0, 12 * (size_t)V, s));
    const GridD g = to_dev(gh);
    if (M > 0) {
        k_sample_adjoint<<<(M + 255) / 256, 256, 0, s>>>(g, pts, M, d_samples, w.gsdf);
        RTSDF_LAUNCHED();
    }
    const ShadowArgs sa = make_shadow_args(gh, sp);
    if (P > 0) {
        k_shadow_adjoint<<<(P + 127) / 128, 128, 0, s>>>(sa, sdf, pos, nrm, P, d_vis, w.gsdf, w.gl);
        RTSDF_LAUNCHED();
    }
    FieldArgs fa;
    fa.g = g;
    fa.verts = verts;
    fa.V = V;
    fa.tris = tris;
    fa.T = T;
    fa.mask2 = rp.mask_vox * rp.mask_vox;
    fa.inv_h = 1.0f / gh.h;
    fa.k0 = rp.key[0];
    fa.k1 = rp.key[1];
    fa.scene = rp.scene_id;
    fa.fallback = rp.sign_fallback;
    const int64_t want = (int64_t)(nvox + 255) / 256, cap = (int64_t)num_sms() * 16;
    const int64_t blocks = want < cap ? want : cap;
    k_field_adjoint<<<(unsigned)blocks, 256, 0, s>>>(fa, nearest, rep_tri, front, back, win_ray, win_tri, w.gsdf,
                                                     d_verts);
    RTSDF_LAUNCHED();
    const float* l = sp.light_dir;
    const float len = sp.light_dir_device ? 0.0f : sqrtf(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    k_light_finalize<<<1, 32, 0, s>>>(w.gl, sa.L, len, sp.light_dir_device, d_light);
    RTSDF_LAUNCHED();
    return RTSDF_OK;
}

}  // namespace rtsdf
