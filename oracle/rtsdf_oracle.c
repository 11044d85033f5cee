/*
 * CPU oracle of the RTSDF hot path -- TEST INFRASTRUCTURE ONLY (see rtsdf_oracle.h).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (never -ffast-math).
 * Every expression below is evaluated in the order written, in IEEE FP32, with
 * correctly rounded division and square root, so each integer decision taken
 * from floating point is reproducible by any implementation that performs the
 * same operations.  OpenMP only splits independent voxels or pixels; results do
 * not depend on the thread count.
 */
#include "rtsdf_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- vectors */

static inline float dot3(const float* x, const float* y) {
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}
static inline void sub3(const float* x, const float* y, float* r) {
    r[0] = x[0] - y[0];
    r[1] = x[1] - y[1];
    r[2] = x[2] - y[2];
}
static inline void cross3(const float* x, const float* y, float* r) {
    r[0] = x[1] * y[2] - x[2] * y[1];
    r[1] = x[2] * y[0] - x[0] * y[2];
    r[2] = x[0] * y[1] - x[1] * y[0];
}
static inline uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}
static inline float bitsf(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

void or_to_voxel(const float* verts, int32_t V, const or_grid* g, float* out) {
    for (int64_t i = 0; i < V; ++i) {
        out[3 * i + 0] = (verts[3 * i + 0] - g->ox) / g->h;
        out[3 * i + 1] = (verts[3 * i + 1] - g->oy) / g->h;
        out[3 * i + 2] = (verts[3 * i + 2] - g->oz) / g->h;
    }
}

/* A triangle takes part only if its three indices address vertices and all nine
 * voxel-space coordinates are finite; other triangles are skipped everywhere. */
static int tri_valid(const float* vv, int32_t V, const int32_t* tris, int32_t t) {
    for (int c = 0; c < 3; ++c) {
        int32_t id = tris[3 * (int64_t)t + c];
        if (id < 0 || id >= V) return 0;
        for (int a = 0; a < 3; ++a)
            if (!isfinite(vv[3 * (int64_t)id + a])) return 0;
    }
    return 1;
}

/* ------------------------------------------------- triangle / box overlap */

/* Separating-axis theorem for a closed triangle and a closed cube.  Candidate
 * axes: the three box normals, the triangle normal and the nine cross products
 * of a triangle edge with a box normal.  The sets are disjoint iff on some axis
 * the projected triangle interval lies strictly outside [-r, r]. */
int or_tri_box_overlap(const float* a, const float* b, const float* c,
                       float cx, float cy, float cz, float hs) {
    const float cen[3] = {cx, cy, cz};
    float v[3][3];
    sub3(a, cen, v[0]);
    sub3(b, cen, v[1]);
    sub3(c, cen, v[2]);

    /* box normals: the triangle's bounding interval on each axis */
    for (int ax = 0; ax < 3; ++ax) {
        float mn = fminf(fminf(v[0][ax], v[1][ax]), v[2][ax]);
        float mx = fmaxf(fmaxf(v[0][ax], v[1][ax]), v[2][ax]);
        if (mn > hs || mx < -hs) return 0;
    }

    float e[3][3];
    sub3(v[1], v[0], e[0]);
    sub3(v[2], v[1], e[1]);
    sub3(v[0], v[2], e[2]);

    /* triangle normal: plane n.x = n.v0 against the box's support radius */
    float n[3];
    cross3(e[0], e[1], n);
    {
        float d = dot3(n, v[0]);
        float r = hs * (fabsf(n[0]) + fabsf(n[1]) + fabsf(n[2]));
        if (d > r || d < -r) return 0;
    }

    /* edge x box-normal axes.  e x X = (0, e.z, -e.y), e x Y = (-e.z, 0, e.x),
     * e x Z = (e.y, -e.x, 0); each projection uses the two non-zero components. */
    for (int i = 0; i < 3; ++i) {
        const float* E = e[i];
        for (int ax = 0; ax < 3; ++ax) {
            int p = (ax + 1) % 3, q = (ax + 2) % 3; /* the two live components */
            float ap, aq;
            if (ax == 0) { ap = E[2]; aq = -E[1]; }        /* (y, z) */
            else if (ax == 1) { ap = E[0]; aq = -E[2]; }   /* (z, x): a = (-e.z, 0, e.x) */
            else { ap = E[1]; aq = -E[0]; }                /* (x, y) */
            float p0 = v[0][p] * ap + v[0][q] * aq;
            float p1 = v[1][p] * ap + v[1][q] * aq;
            float p2 = v[2][p] * ap + v[2][q] * aq;
            float mn = fminf(fminf(p0, p1), p2);
            float mx = fmaxf(fmaxf(p0, p1), p2);
            float r = hs * (fabsf(ap) + fabsf(aq));
            if (mn > r || mx < -r) return 0;
        }
    }
    return 1;
}

/* ------------------------------------------------ closest point on triangle */

/* Walk the Voronoi regions of the triangle (vertices, edges, face) as in Ericson,
 * Real-Time Collision Detection, Sec. 5.1.5, in the frame where p is the origin. */
float or_closest_d2(const float* p, const float* A, const float* B, const float* C) {
    float a[3], b[3], c[3], ab[3], ac[3], q[3];
    sub3(A, p, a);
    sub3(B, p, b);
    sub3(C, p, c);
    sub3(b, a, ab);
    sub3(c, a, ac);
    const float pa[3] = {-a[0], -a[1], -a[2]}; /* p - a */
    float d1 = dot3(ab, pa), d2 = dot3(ac, pa);
    if (d1 <= 0.0f && d2 <= 0.0f) return dot3(a, a);

    const float pb[3] = {-b[0], -b[1], -b[2]};
    float d3 = dot3(ab, pb), d4 = dot3(ac, pb);
    if (d3 >= 0.0f && d4 <= d3) return dot3(b, b);

    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        float s = d1 / (d1 - d3);
        q[0] = a[0] + s * ab[0];
        q[1] = a[1] + s * ab[1];
        q[2] = a[2] + s * ab[2];
        return dot3(q, q);
    }

    const float pc[3] = {-c[0], -c[1], -c[2]};
    float d5 = dot3(ab, pc), d6 = dot3(ac, pc);
    if (d6 >= 0.0f && d5 <= d6) return dot3(c, c);

    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        float s = d2 / (d2 - d6);
        q[0] = a[0] + s * ac[0];
        q[1] = a[1] + s * ac[1];
        q[2] = a[2] + s * ac[2];
        return dot3(q, q);
    }

    float va = d3 * d6 - d5 * d4;
    float e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
        float s = e43 / (e43 + e56);
        float bc[3];
        sub3(c, b, bc);
        q[0] = b[0] + s * bc[0];
        q[1] = b[1] + s * bc[1];
        q[2] = b[2] + s * bc[2];
        return dot3(q, q);
    }

    float inv = 1.0f / (va + vb + vc);
    float sv = vb * inv, sw = vc * inv;
    q[0] = a[0] + ab[0] * sv + ac[0] * sw;
    q[1] = a[1] + ab[1] * sv + ac[1] * sw;
    q[2] = a[2] + ab[2] * sv + ac[2] * sw;
    return dot3(q, q);
}

/* ------------------------------------------------------------ voxelization */

int32_t or_voxelize(const float* vv, int32_t V, const int32_t* tris, int32_t T,
                    const or_grid* g, int32_t* seed, int32_t* rep_tri) {
    const int64_t nvox = (int64_t)g->nx * g->ny * g->nz;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nvox > 0 ? nvox : 1));
    for (int64_t i = 0; i < nvox; ++i) key[i] = UINT64_MAX;
    int32_t skipped = 0;
    const float dims[3] = {(float)g->nx, (float)g->ny, (float)g->nz};

    for (int32_t t = 0; t < T; ++t) {
        if (!tri_valid(vv, V, tris, t)) { ++skipped; continue; }
        const float* a = vv + 3 * (int64_t)tris[3 * (int64_t)t + 0];
        const float* b = vv + 3 * (int64_t)tris[3 * (int64_t)t + 1];
        const float* c = vv + 3 * (int64_t)tris[3 * (int64_t)t + 2];
        /* voxel i spans [i, i+1]; the closed triangle can touch it only if
         * min <= i+1 and max >= i, i.e. i in [ceil(min)-1, floor(max)] */
        int lo[3], hi[3], empty = 0;
        for (int ax = 0; ax < 3; ++ax) {
            float mn = fminf(fminf(a[ax], b[ax]), c[ax]);
            float mx = fmaxf(fmaxf(a[ax], b[ax]), c[ax]);
            float l = fmaxf(ceilf(mn) - 1.0f, 0.0f);
            float h = fminf(floorf(mx), dims[ax] - 1.0f);
            if (l > h) { empty = 1; break; }
            lo[ax] = (int)l;
            hi[ax] = (int)h;
        }
        if (empty) continue;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                    if (!or_tri_box_overlap(a, b, c, p[0], p[1], p[2], 0.5f)) continue;
                    float d2 = or_closest_d2(p, a, b, c);
                    uint64_t kk = ((uint64_t)fbits(d2) << 32) | (uint32_t)t;
                    int64_t lin = ((int64_t)k * g->ny + j) * g->nx + i;
                    if (kk < key[lin]) key[lin] = kk;
                }
    }
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                int64_t lin = ((int64_t)k * g->ny + j) * g->nx + i;
                if (key[lin] == UINT64_MAX) {
                    seed[lin] = OR_EMPTY;
                    rep_tri[lin] = -1;
                } else {
                    seed[lin] = (k << 20) | (j << 10) | i;
                    rep_tri[lin] = (int32_t)(uint32_t)(key[lin] & 0xffffffffu);
                }
            }
    free(key);
    return skipped;
}

/* ------------------------------------------------------------ jump flooding */

static inline int32_t seed_d2(int i, int j, int k, int32_t s) {
    int dx = i - (s & 1023), dy = j - ((s >> 10) & 1023), dz = k - ((s >> 20) & 1023);
    return dx * dx + dy * dy + dz * dz;
}

void or_jfa_pass(const or_grid* g, const int32_t* in, int32_t step, int32_t* out) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int32_t best = OR_EMPTY, bd = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int x = i + dx * step, y = j + dy * step, z = k + dz * step;
                            if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                            int32_t s = in[((int64_t)z * ny + y) * nx + x];
                            if (s == OR_EMPTY) continue;
                            int32_t d = seed_d2(i, j, k, s);
                            if (best == OR_EMPTY || d < bd || (d == bd && s < best)) {
                                best = s;
                                bd = d;
                            }
                        }
                out[((int64_t)k * ny + j) * nx + i] = best;
            }
}

/* ---------------------------------------------------------------- resolve */

void or_resolve(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                const int32_t* rep_tri, float mask_vox, float empty_dist,
                float* u_c, uint8_t* mask) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const float m2 = mask_vox * mask_vox;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t lin = ((int64_t)k * ny + j) * nx + i;
                int32_t s = nearest[lin];
                int32_t rep = -1;
                if (s != OR_EMPTY) {
                    int64_t sl = ((int64_t)((s >> 20) & 1023) * ny + ((s >> 10) & 1023)) * nx + (s & 1023);
                    rep = rep_tri[sl];
                }
                if (rep < 0) {
                    u_c[lin] = empty_dist;
                    mask[lin] = 0;
                    continue;
                }
                float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                const int32_t* tr = tris + 3 * (int64_t)rep;
                u_c[lin] = sqrtf(or_closest_d2(p, vv + 3 * (int64_t)tr[0], vv + 3 * (int64_t)tr[1],
                                               vv + 3 * (int64_t)tr[2]));
                mask[lin] = ((float)seed_d2(i, j, k, s) <= m2) ? 1 : 0;
            }
}

/* Two resolutions (Sec. 2.5.1: the coarse SDF by jump flooding at 128^3, the fine
 * SDF at 256^3): fine voxel (i,j,k) lies in coarse voxel (i/r, j/r, k/r); its
 * flooded seed and representative triangle are that coarse voxel's; the distance
 * is measured from the fine voxel's centre (vv in fine voxel units); the mask
 * compares the integer seed distance in coarse voxels. */
void or_resolve_2res(const or_grid* gf, const or_grid* gc, int32_t ratio, const float* vv, const int32_t* tris,
                     const int32_t* nearest_c, const int32_t* rep_c, float mask_vox, float empty_dist, float* u_c,
                     uint8_t* mask) {
    const int nx = gf->nx, ny = gf->ny, nz = gf->nz;
    const float m2 = mask_vox * mask_vox;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t lin = ((int64_t)k * ny + j) * nx + i;
                const int ic = i / ratio, jc = j / ratio, kc = k / ratio;
                const int32_t s = nearest_c[((int64_t)kc * gc->ny + jc) * gc->nx + ic];
                int32_t rep = -1;
                if (s != OR_EMPTY)
                    rep = rep_c[((int64_t)((s >> 20) & 1023) * gc->ny + ((s >> 10) & 1023)) * gc->nx + (s & 1023)];
                if (rep < 0) {
                    u_c[lin] = empty_dist;
                    mask[lin] = 0;
                    continue;
                }
                const float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                const int32_t* tr = tris + 3 * (int64_t)rep;
                u_c[lin] = sqrtf(or_closest_d2(p, vv + 3 * (int64_t)tr[0], vv + 3 * (int64_t)tr[1],
                                               vv + 3 * (int64_t)tr[2]));
                mask[lin] = ((float)seed_d2(ic, jc, kc, s) <= m2) ? 1 : 0;
            }
}

/* The representative triangle each fine voxel's sign fallback uses (that of its
 * coarse voxel's flooded seed), as a fine grid. */
void or_fine_rep_2res(const or_grid* gf, const or_grid* gc, int32_t ratio, const int32_t* nearest_c,
                      const int32_t* rep_c, int32_t* rep_f) {
    const int nx = gf->nx, ny = gf->ny, nz = gf->nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int32_t s = nearest_c[((int64_t)(k / ratio) * gc->ny + j / ratio) * gc->nx + i / ratio];
                rep_f[((int64_t)k * ny + j) * nx + i] =
                    s == OR_EMPTY ? -1
                                  : rep_c[((int64_t)((s >> 20) & 1023) * gc->ny + ((s >> 10) & 1023)) * gc->nx +
                                          (s & 1023)];
            }
}

/* ------------------------------------------------------------------ Philox */

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two
 * round constants, swaps the halves and mixes in the key; the key is advanced by
 * the two Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t m0 = (uint64_t)0xD2511F53u * c0;
        uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)m1;
        uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)m0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Marsaglia's method: draw (u, v) uniform in [-1, 1)^2, keep it when
 * 0 < s = u^2 + v^2 < 1, and map to (2u sqrt(1-s), 2v sqrt(1-s), 1 - 2s), which is
 * uniform on the sphere.  Each Philox call gives two candidate pairs; the attempt
 * number is the fourth counter word.  u = (x >> 8) * 2^-23 - 1 is exact. */
int or_sphere_dir(uint32_t voxel, uint32_t ray, uint32_t scene, const uint32_t key[2], float dir[3]) {
    for (uint32_t att = 0; att < 32; ++att) {
        const uint32_t ctr[4] = {voxel, ray, scene, att};
        uint32_t x[4];
        or_philox4x32_10(ctr, key, x);
        for (int pr = 0; pr < 2; ++pr) {
            float u = (float)(x[2 * pr] >> 8) * 0x1p-23f - 1.0f;
            float v = (float)(x[2 * pr + 1] >> 8) * 0x1p-23f - 1.0f;
            float s = u * u + v * v;
            if (s > 0.0f && s < 1.0f) {
                float a = 2.0f * sqrtf(1.0f - s);
                dir[0] = u * a;
                dir[1] = v * a;
                dir[2] = 1.0f - 2.0f * s;
                return (int)att;
            }
        }
    }
    return -1;
}

/* -------------------------------------------------------- ray / triangle */

int or_ray_tri(const float o[3], const float d[3], const float* A, const float* B, const float* C,
               float tmax, float* t, int* front, float* margin) {
    float e1[3], e2[3], p[3], tv[3], q[3];
    sub3(B, A, e1);
    sub3(C, A, e2);
    cross3(d, e2, p);
    float det = dot3(e1, p);
    if (det == 0.0f) return 0;
    float inv = 1.0f / det;
    sub3(o, A, tv);
    float u = dot3(tv, p) * inv;
    if (u < 0.0f || u > 1.0f) return 0;
    cross3(tv, e1, q);
    float w = dot3(d, q) * inv;
    float uw = u + w;
    if (w < 0.0f || uw > 1.0f) return 0;
    float tt = dot3(e2, q) * inv;
    if (!(tt > 0.0f && tt <= tmax)) return 0;
    *t = tt;
    *front = det > 0.0f; /* det = -d.(e1 x e2): positive when the ray faces the outward normal */
    if (margin) {
        float m = u < w ? u : w;
        float r = 1.0f - uw;
        *margin = m < r ? m : r;
    }
    return 1;
}

/* ------------------------------------------------------------- refinement */

int64_t or_refine_voxels(const or_grid* g, const float* vv, int32_t V, const int32_t* tris, int32_t T,
                         const int32_t* vox, int64_t n, int32_t R, float tmax,
                         const uint32_t key[2], uint32_t frame, uint32_t scene,
                         uint32_t* dist_bits, uint32_t* front, uint32_t* back,
                         uint32_t* win_ray, int32_t* win_tri, int64_t* near_edge) {
    uint8_t* ok = (uint8_t*)malloc((size_t)(T > 0 ? T : 1));
    for (int32_t t = 0; t < T; ++t) ok[t] = (uint8_t)tri_valid(vv, V, tris, t);
    int64_t failed = 0, near = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : failed, near)
    for (int64_t n_i = 0; n_i < n; ++n_i) {
        int32_t lin = vox[n_i];
        int i = lin % g->nx, j = (lin / g->nx) % g->ny, k = lin / (g->nx * g->ny);
        const float o[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
        float dist = bitsf(dist_bits[lin]);
        uint32_t fr = front[lin], bk = back[lin];
        /* closest hit over this call's rays: (t, triangle) ordered, first ray on ties */
        float fbest = INFINITY;
        int32_t fbest_tri = -1;
        uint32_t fbest_ray = 0xFFFFFFFFu;
        for (int32_t r = 0; r < R; ++r) {
            float dir[3];
            const uint32_t ray = frame * (uint32_t)R + (uint32_t)r;
            if (or_sphere_dir((uint32_t)lin, ray, scene, key, dir) < 0) {
                ++failed;
                continue;
            }
            float best = INFINITY;
            int best_front = 0, hit = 0;
            int32_t best_tri = -1;
            for (int32_t t = 0; t < T; ++t) {
                if (!ok[t]) continue;
                const int32_t* tr = tris + 3 * (int64_t)t;
                float tt, margin;
                int f;
                if (!or_ray_tri(o, dir, vv + 3 * (int64_t)tr[0], vv + 3 * (int64_t)tr[1],
                                vv + 3 * (int64_t)tr[2], tmax, &tt, &f, &margin))
                    continue;
                if (margin < 1e-6f) ++near;
                if (tt < best) { /* ascending ids: strict < keeps the lower id on ties */
                    best = tt;
                    best_front = f;
                    best_tri = t;
                    hit = 1;
                }
            }
            if (hit) {
                if (best < fbest || (best == fbest && best_tri < fbest_tri)) {
                    fbest = best;
                    fbest_tri = best_tri;
                    fbest_ray = ray;
                }
                if (best_front) ++fr; else ++bk;
            }
        }
        if (fbest < dist) {
            dist = fbest;
            if (win_ray) win_ray[lin] = fbest_ray;
            if (win_tri) win_tri[lin] = fbest_tri;
        }
        dist_bits[lin] = fbits(dist);
        front[lin] = fr;
        back[lin] = bk;
    }
    free(ok);
    if (near_edge) *near_edge = near;
    return failed;
}

int or_vote_sign(uint32_t front, uint32_t back, const float* p, const float* a, const float* b,
                 const float* c, int fallback) {
    if (back > front) return -1;
    if (front > back || !fallback) return 1;
    float e1[3], e2[3], nrm[3], pa[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, nrm);
    sub3(p, a, pa);
    return dot3(pa, nrm) < 0.0f ? -1 : 1;
}

void or_finalize(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                 const int32_t* rep_tri, const uint8_t* mask, const float* u_c,
                 const uint32_t* dist_bits, const uint32_t* front, const uint32_t* back,
                 float beta, int fallback, float* sdf) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t lin = ((int64_t)k * ny + j) * nx + i;
                if (!mask[lin]) {
                    sdf[lin] = u_c[lin] - beta;
                    continue;
                }
                int32_t s = nearest[lin];
                int64_t sl = ((int64_t)((s >> 20) & 1023) * ny + ((s >> 10) & 1023)) * nx + (s & 1023);
                const int32_t* tr = tris + 3 * (int64_t)rep_tri[sl];
                const float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                int sg = or_vote_sign(front[lin], back[lin], p, vv + 3 * (int64_t)tr[0],
                                      vv + 3 * (int64_t)tr[1], vv + 3 * (int64_t)tr[2], fallback);
                float d = bitsf(dist_bits[lin]);
                sdf[lin] = sg < 0 ? -d : d;
            }
}

/* -------------------------------------------------------------- raymarch */

static inline float lerpf(float a, float b, float t) { return a + (b - a) * t; }

float or_trilinear(const or_grid* g, const float* sdf, float qx, float qy, float qz) {
    const float s[3] = {qx - 0.5f, qy - 0.5f, qz - 0.5f};
    const int n[3] = {g->nx, g->ny, g->nz};
    int i0[3], i1[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
        float fl = floorf(s[a]);
        f[a] = s[a] - fl;
        int lo = (int)fl, hi = lo + 1;
        i0[a] = lo < 0 ? 0 : (lo > n[a] - 1 ? n[a] - 1 : lo);
        i1[a] = hi < 0 ? 0 : (hi > n[a] - 1 ? n[a] - 1 : hi);
    }
#define AT(x, y, z) sdf[((int64_t)(z) * g->ny + (y)) * g->nx + (x)]
    float c00 = lerpf(AT(i0[0], i0[1], i0[2]), AT(i1[0], i0[1], i0[2]), f[0]);
    float c10 = lerpf(AT(i0[0], i1[1], i0[2]), AT(i1[0], i1[1], i0[2]), f[0]);
    float c01 = lerpf(AT(i0[0], i0[1], i1[2]), AT(i1[0], i0[1], i1[2]), f[0]);
    float c11 = lerpf(AT(i0[0], i1[1], i1[2]), AT(i1[0], i1[1], i1[2]), f[0]);
#undef AT
    float c0 = lerpf(c00, c10, f[1]);
    float c1 = lerpf(c01, c11, f[1]);
    return lerpf(c0, c1, f[2]);
}

void or_sample(const or_grid* g, const float* sdf, const float* pts, int32_t M, float* out) {
    for (int32_t m = 0; m < M; ++m) {
        const float* p = pts + 3 * (int64_t)m;
        out[m] = or_trilinear(g, sdf, (p[0] - g->ox) / g->h, (p[1] - g->oy) / g->h, (p[2] - g->oz) / g->h);
    }
}

/* Sphere tracing toward the light (Sec. 2.4) with the penumbra estimate
 * k * (closest approach) / (distance along the ray), where the closest approach
 * between two successive samples is triangulated from the two sampled distances
 * (Sec. 2.5.2, after Aaltonen 2018): y = d^2 / (2 d_prev), e = sqrt(d^2 - y^2).
 * Steps are capped at max_step (Sec. 2.5.2); the march starts start_off along
 * the ray from a point lifted normal_off along the normal (Sec. 2.5.3), and the
 * SDF is thickened by bias (Sec. 2.5.3). */
/* Jittered first-sample distances (Sec. 2.5.2: the ray's offset moves slightly
 * along the light): t_i = start_off + jitter * u_i, u_i the top 24 bits of the first
 * word of Philox4x32-10 on counter (i, frame, 0x4A177E2, 0), key (0x51AD0, 0x7E2),
 * times 2^-24. */
void or_jitter_starts(int32_t P, float start_off, float jitter, uint32_t frame, float* t_start) {
    const uint32_t key[2] = {0x51AD0u, 0x7E2u};
    for (int32_t i = 0; i < P; ++i) {
        const uint32_t ctr[4] = {(uint32_t)i, frame, 0x4A177E2u, 0u};
        uint32_t x[4];
        or_philox4x32_10(ctr, key, x);
        const float u = (float)(x[0] >> 8) * 0x1p-24f;
        t_start[i] = jitter == 0.0f ? start_off : start_off + jitter * u;
    }
}

void or_shadow(const or_grid* g, const float* sdf, const float* pos, const float* nrm, int32_t P,
               const float light_dir[3], float k, int32_t steps, float max_step, float start_off,
               float normal_off, float hit_eps, float bias, const float* t_start, float* vis) {
    float len = sqrtf(dot3(light_dir, light_dir));
    const float L[3] = {light_dir[0] / len, light_dir[1] / len, light_dir[2] / len};
    const float nxf = (float)g->nx, nyf = (float)g->ny, nzf = (float)g->nz;
#pragma omp parallel for schedule(static)
    for (int32_t pi = 0; pi < P; ++pi) {
        const float* x = pos + 3 * (int64_t)pi;
        const float* n = nrm + 3 * (int64_t)pi;
        float org[3];
        org[0] = (x[0] - g->ox) / g->h + normal_off * n[0];
        org[1] = (x[1] - g->oy) / g->h + normal_off * n[1];
        org[2] = (x[2] - g->oz) / g->h + normal_off * n[2];
        float t = t_start ? t_start[pi] : start_off, res = 1.0f, d_prev = INFINITY;
        for (int32_t s = 0; s < steps; ++s) {
            float qx = org[0] + t * L[0], qy = org[1] + t * L[1], qz = org[2] + t * L[2];
            if (qx < 0.0f || qx > nxf || qy < 0.0f || qy > nyf || qz < 0.0f || qz > nzf) break;
            float d = or_trilinear(g, sdf, qx, qy, qz) - bias;
            if (d <= hit_eps) {
                res = 0.0f;
                break;
            }
            float dd = d * d;
            float y = dd / (2.0f * d_prev);
            float e = sqrtf(fmaxf(dd - y * y, 0.0f));
            res = fminf(res, (k * e) / fmaxf(t - y, 1e-6f));
            d_prev = d;
            t = t + fminf(d, max_step);
        }
        vis[pi] = fminf(fmaxf(res, 0.0f), 1.0f);
    }
}
