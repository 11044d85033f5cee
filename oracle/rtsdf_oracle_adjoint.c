/*
 * FP64 reference of the adjoint of the RTSDF field and shadow with frozen
 * discrete choices -- TEST INFRASTRUCTURE ONLY (see rtsdf_oracle.h).
 *
 * The differentiable function: every discrete choice of the FP32 forward is held
 * fixed (the flooded seed and its representative triangle, the ray mask, the
 * vote sign, which source won a refined distance -- the coarse closest point or
 * one ray's hit -- and the raymarch's control flow: its stop step, the branch of
 * every step cap, the sample that attains the penumbra minimum and the trilinear
 * cell of every sample).  With those frozen, the field and the losses are smooth
 * functions of the vertex positions and the light direction, evaluated here in
 * FP64; their gradients follow by the envelope theorem for the closest point
 * (d|p - q|/dX_m = lambda_m (q - p)/|p - q|), implicit differentiation of the
 * ray/plane hit (dt/dX_m = lambda_m n / (n.d)), and reverse-mode differentiation
 * of the sample and raymarch formulas.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "rtsdf_oracle.h"

static inline double d_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void d_sub(const double* a, const double* b, double* r) {
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}
static inline void d_cross(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------ frozen sources */

void or_frozen_sources(const or_grid* g, const float* vv, const int32_t* tris, const int32_t* nearest,
                       const int32_t* rep_tri, const uint8_t* mask, const uint32_t* front, const uint32_t* back,
                       const uint32_t* win_ray, const int32_t* win_tri, const uint32_t key[2], uint32_t scene,
                       int fallback, or_src* out) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t lin = ((int64_t)k * ny + j) * nx + i;
                or_src* s = out + lin;
                memset(s, 0, sizeof(*s));
                const int32_t sd = nearest[lin];
                int32_t rep = -1;
                if (sd != OR_EMPTY) {
                    const int64_t sl = ((int64_t)((sd >> 20) & 1023) * ny + ((sd >> 10) & 1023)) * nx + (sd & 1023);
                    rep = rep_tri[sl];
                }
                if (rep < 0) {
                    s->kind = OR_SRC_CONST;
                    s->tri = -1;
                    continue;
                }
                s->tri = rep;
                s->sign = 1.0f;
                if (!mask[lin]) {
                    s->kind = OR_SRC_COARSE_UNMASKED;
                    continue;
                }
                const float p[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                const int32_t* tr = tris + 3 * (int64_t)rep;
                s->sign = (float)or_vote_sign(front[lin], back[lin], p, vv + 3 * (int64_t)tr[0],
                                              vv + 3 * (int64_t)tr[1], vv + 3 * (int64_t)tr[2], fallback);
                if (win_ray[lin] == 0xFFFFFFFFu) {
                    s->kind = OR_SRC_COARSE_MASKED;
                } else {
                    s->kind = OR_SRC_RAY;
                    s->tri = win_tri[lin];
                    or_sphere_dir((uint32_t)lin, win_ray[lin], scene, key, s->dir);
                }
            }
}

/* closest point of triangle abc to p in FP64, with its barycentric weights */
static void closest_point_f64(const double* p, const double* A, const double* B, const double* C, double q[3],
                              double lam[3]) {
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    d_sub(B, A, ab);
    d_sub(C, A, ac);
    d_sub(p, A, ap);
    const double d1 = d_dot(ab, ap), d2 = d_dot(ac, ap);
    double la = 1, lb = 0, lc = 0;
    if (d1 <= 0 && d2 <= 0) goto done;
    d_sub(p, B, bp);
    {
        const double d3 = d_dot(ab, bp), d4 = d_dot(ac, bp);
        if (d3 >= 0 && d4 <= d3) { la = 0; lb = 1; goto done; }
        const double vc = d1 * d4 - d3 * d2;
        if (vc <= 0 && d1 >= 0 && d3 <= 0) { const double v = d1 / (d1 - d3); la = 1 - v; lb = v; goto done; }
        d_sub(p, C, cp);
        const double d5 = d_dot(ab, cp), d6 = d_dot(ac, cp);
        if (d6 >= 0 && d5 <= d6) { la = 0; lc = 1; goto done; }
        const double vb = d5 * d2 - d1 * d6;
        if (vb <= 0 && d2 >= 0 && d6 <= 0) { const double w = d2 / (d2 - d6); la = 1 - w; lc = w; goto done; }
        const double va = d3 * d6 - d5 * d4;
        if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
            const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
            la = 0; lb = 1 - w; lc = w;
            goto done;
        }
        const double den = 1.0 / (va + vb + vc);
        lb = vb * den;
        lc = vc * den;
        la = 1 - lb - lc;
    }
done:
    for (int a = 0; a < 3; ++a) q[a] = la * A[a] + lb * B[a] + lc * C[a];
    lam[0] = la;
    lam[1] = lb;
    lam[2] = lc;
}

static void vox64(const or_grid* g, const double* verts, int32_t id, double out[3]) {
    const double o[3] = {g->ox, g->oy, g->oz};
    for (int a = 0; a < 3; ++a) out[a] = (verts[3 * (int64_t)id + a] - o[a]) / (double)g->h;
}

/* Value of one voxel's frozen field (voxel units) and, when gv != NULL, adds
 * g * d(value)/d(world vertex) into gv. */
static double frozen_voxel(const or_grid* g, const double* verts, const int32_t* tris, const or_src* s, int i, int j,
                           int k, double beta, double g_in, double* gv) {
    if (s->kind == OR_SRC_CONST) return (double)(g->nx + g->ny + g->nz) - beta;
    const int32_t* tr = tris + 3 * (int64_t)s->tri;
    double X[3][3];
    for (int m = 0; m < 3; ++m) vox64(g, verts, tr[m], X[m]);
    const double p[3] = {i + 0.5, j + 0.5, k + 0.5};
    const double inv_h = 1.0 / (double)g->h;
    if (s->kind != OR_SRC_RAY) {
        double q[3], lam[3], pq[3];
        closest_point_f64(p, X[0], X[1], X[2], q, lam);
        d_sub(q, p, pq);
        const double u = sqrt(d_dot(pq, pq));
        const double sg = s->kind == OR_SRC_COARSE_UNMASKED ? 1.0 : (double)s->sign;
        if (gv && u > 0)
            for (int m = 0; m < 3; ++m)
                for (int a = 0; a < 3; ++a) gv[3 * (int64_t)tr[m] + a] += g_in * sg * lam[m] * pq[a] / u * inv_h;
        return s->kind == OR_SRC_COARSE_UNMASKED ? u - beta : sg * u;
    }
    const double d[3] = {s->dir[0], s->dir[1], s->dir[2]};
    double e1[3], e2[3], n[3], ao[3];
    d_sub(X[1], X[0], e1);
    d_sub(X[2], X[0], e2);
    d_cross(e1, e2, n);
    d_sub(X[0], p, ao);
    const double dn = d_dot(d, n);
    const double t = d_dot(ao, n) / dn;
    if (gv) {
        /* barycentric weights of the hit point P = p + t d */
        const double P[3] = {p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]};
        double ap[3], c1[3], c2[3];
        d_sub(P, X[0], ap);
        d_cross(ap, e2, c1);
        d_cross(e1, ap, c2);
        const double nn = d_dot(n, n);
        const double lb = d_dot(c1, n) / nn, lc = d_dot(c2, n) / nn, la = 1 - lb - lc;
        const double lam[3] = {la, lb, lc};
        for (int m = 0; m < 3; ++m)
            for (int a = 0; a < 3; ++a)
                gv[3 * (int64_t)tr[m] + a] += g_in * (double)s->sign * lam[m] * n[a] / dn * inv_h;
    }
    return (double)s->sign * t;
}

void or_frozen_sdf_f64(const or_grid* g, const double* verts, const int32_t* tris, const or_src* src, double beta,
                       double* sdf) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t lin = ((int64_t)k * ny + j) * nx + i;
                sdf[lin] = frozen_voxel(g, verts, tris, src + lin, i, j, k, beta, 0.0, NULL);
            }
}

void or_frozen_sdf_backward_f64(const or_grid* g, const double* verts, const int32_t* tris, const or_src* src,
                                double beta, const double* gsdf, double* gverts) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    /* sequential: scattered accumulation into shared vertices */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t lin = ((int64_t)k * ny + j) * nx + i;
                if (gsdf[lin] != 0.0) frozen_voxel(g, verts, tris, src + lin, i, j, k, beta, gsdf[lin], gverts);
            }
}

/* ------------------------------------------------------------ trilinear (FP64) */

typedef struct {
    int64_t c[8];   /* corner linear indices, x fastest: 000,100,010,110,001,101,011,111 */
    double f[3];    /* fractional position in the cell */
    int dead[3];    /* axis clamped to one sample: no derivative along it */
} cell64;

/* cell of voxel coordinate q (clamp to edge); the cell can be given frozen by
 * passing base >= 0 values in fixed_i0 (then only the fractions are recomputed) */
static void cell_of(const or_grid* g, const double q[3], const int fixed_i0[3], cell64* c) {
    const int n[3] = {g->nx, g->ny, g->nz};
    int i0[3], i1[3];
    for (int a = 0; a < 3; ++a) {
        const double s = q[a] - 0.5;
        const int lo = fixed_i0 ? fixed_i0[a] : (int)floor(s);
        c->f[a] = s - lo;
        i0[a] = lo < 0 ? 0 : (lo > n[a] - 1 ? n[a] - 1 : lo);
        i1[a] = lo + 1 < 0 ? 0 : (lo + 1 > n[a] - 1 ? n[a] - 1 : lo + 1);
        c->dead[a] = i0[a] == i1[a];
    }
    for (int b = 0; b < 8; ++b) {
        const int x = (b & 1) ? i1[0] : i0[0], y = (b & 2) ? i1[1] : i0[1], z = (b & 4) ? i1[2] : i0[2];
        c->c[b] = ((int64_t)z * g->ny + y) * g->nx + x;
    }
}

static double tri_value(const cell64* c, const double* f) {
    double v[8];
    for (int b = 0; b < 8; ++b) v[b] = f[c->c[b]];
    const double fx = c->f[0], fy = c->f[1], fz = c->f[2];
    const double c00 = v[0] + (v[1] - v[0]) * fx, c10 = v[2] + (v[3] - v[2]) * fx;
    const double c01 = v[4] + (v[5] - v[4]) * fx, c11 = v[6] + (v[7] - v[6]) * fx;
    const double c0 = c00 + (c10 - c00) * fy, c1 = c01 + (c11 - c01) * fy;
    return c0 + (c1 - c0) * fz;
}

/* weights of the 8 corners and the gradient of the interpolant w.r.t. q */
static void tri_weights(const cell64* c, const double* f, double w[8], double grad[3]) {
    const double fx = c->f[0], fy = c->f[1], fz = c->f[2];
    for (int b = 0; b < 8; ++b)
        w[b] = ((b & 1) ? fx : 1 - fx) * ((b & 2) ? fy : 1 - fy) * ((b & 4) ? fz : 1 - fz);
    if (!grad) return;
    double v[8];
    for (int b = 0; b < 8; ++b) v[b] = f[c->c[b]];
    grad[0] = grad[1] = grad[2] = 0;
    for (int b = 0; b < 8; ++b) {
        const double wx = (b & 1) ? 1 : -1, wy = (b & 2) ? 1 : -1, wz = (b & 4) ? 1 : -1;
        grad[0] += v[b] * wx * ((b & 2) ? fy : 1 - fy) * ((b & 4) ? fz : 1 - fz);
        grad[1] += v[b] * wy * ((b & 1) ? fx : 1 - fx) * ((b & 4) ? fz : 1 - fz);
        grad[2] += v[b] * wz * ((b & 1) ? fx : 1 - fx) * ((b & 2) ? fy : 1 - fy);
    }
    for (int a = 0; a < 3; ++a)
        if (c->dead[a]) grad[a] = 0;
}

double or_sample_loss_f64(const or_grid* g, const double* sdf, const float* pts, int32_t M, const float* target,
                          double* gsdf) {
    double loss = 0;
    for (int32_t m = 0; m < M; ++m) {
        const double q[3] = {((double)pts[3 * m] - g->ox) / g->h, ((double)pts[3 * m + 1] - g->oy) / g->h,
                             ((double)pts[3 * m + 2] - g->oz) / g->h};
        cell64 c;
        cell_of(g, q, NULL, &c);
        const double r = tri_value(&c, sdf) - (double)target[m];
        loss += r * r;
        if (gsdf) {
            double w[8];
            tri_weights(&c, sdf, w, NULL);
            for (int b = 0; b < 8; ++b) gsdf[c.c[b]] += 2 * r * w[b];
        }
    }
    return loss;
}

/* ------------------------------------------------------------ shadow (frozen) */

#define OR_MAX_STEPS 512

double or_shadow_loss_f64(const or_grid* g, const float* sdf32, const double* sdf, const float* pos,
                          const float* nrm, int32_t P, const float l_decide[3], const double l[3], float k,
                          int32_t steps, float max_step, float start_off, float normal_off, float hit_eps,
                          float bias, const float* t_start, const float* target, double* gsdf, double* gl) {
    /* FP32 light as the forward normalises it: the control flow comes from there */
    const float lf[3] = {l_decide[0], l_decide[1], l_decide[2]};
    const float lenf = sqrtf(lf[0] * lf[0] + lf[1] * lf[1] + lf[2] * lf[2]);
    const float L32[3] = {lf[0] / lenf, lf[1] / lenf, lf[2] / lenf};
    const double len = sqrt(d_dot(l, l));
    const double L[3] = {l[0] / len, l[1] / len, l[2] / len};
    const float nxf = (float)g->nx, nyf = (float)g->ny, nzf = (float)g->nz;
    double loss = 0, gL[3] = {0, 0, 0};
    int32_t ns = steps < OR_MAX_STEPS ? steps : OR_MAX_STEPS;
    for (int32_t pi = 0; pi < P; ++pi) {
        const float* x = pos + 3 * (int64_t)pi;
        const float* n = nrm + 3 * (int64_t)pi;
        /* --- FP32 forward: decisions */
        float org32[3];
        org32[0] = (x[0] - g->ox) / g->h + normal_off * n[0];
        org32[1] = (x[1] - g->oy) / g->h + normal_off * n[1];
        org32[2] = (x[2] - g->oz) / g->h + normal_off * n[2];
        const float t0 = t_start ? t_start[pi] : start_off;
        float t32 = t0, res32 = 1.0f, dprev32 = INFINITY;
        int cells[OR_MAX_STEPS][3];
        unsigned char capped[OR_MAX_STEPS];
        int nsteps = 0, argmin = -1, hit = 0;
        int den_tiny32 = 0, e_pos32 = 0; /* branches of the estimate at the argmin */
        for (int32_t s = 0; s < ns; ++s) {
            const float q[3] = {org32[0] + t32 * L32[0], org32[1] + t32 * L32[1], org32[2] + t32 * L32[2]};
            if (q[0] < 0.0f || q[0] > nxf || q[1] < 0.0f || q[1] > nyf || q[2] < 0.0f || q[2] > nzf) break;
            for (int a = 0; a < 3; ++a) cells[s][a] = (int)floorf(q[a] - 0.5f);
            const float d = or_trilinear(g, sdf32, q[0], q[1], q[2]) - bias;
            nsteps = s + 1;
            if (d <= hit_eps) {
                hit = 1;
                break;
            }
            const float dd = d * d;
            const float y = dd / (2.0f * dprev32);
            const float e = sqrtf(fmaxf(dd - y * y, 0.0f));
            const float r = (k * e) / fmaxf(t32 - y, 1e-6f);
            if (r < res32) {
                res32 = r;
                argmin = s;
                den_tiny32 = !(t32 - y > 1e-6f);
                e_pos32 = dd - y * y > 0.0f;
            }
            dprev32 = d;
            capped[s] = !(d < max_step);
            t32 = t32 + fminf(d, max_step);
        }
        /* --- FP64 values along the frozen path */
        const double tg = (double)target[pi];
        if (hit || argmin < 0 || !(res32 > 0.0f) || !(res32 < 1.0f)) {
            /* the clamped output is constant on the frozen path */
            const double v = (hit || !(res32 > 0.0f)) ? 0.0 : 1.0;
            loss += (v - tg) * (v - tg);
            continue;
        }
        const double org[3] = {((double)x[0] - g->ox) / g->h + (double)normal_off * n[0],
                               ((double)x[1] - g->oy) / g->h + (double)normal_off * n[1],
                               ((double)x[2] - g->oz) / g->h + (double)normal_off * n[2]};
        double tt[OR_MAX_STEPS + 1], dv[OR_MAX_STEPS];
        cell64 cl[OR_MAX_STEPS];
        tt[0] = t0;
        for (int s = 0; s <= argmin; ++s) {
            const double q[3] = {org[0] + tt[s] * L[0], org[1] + tt[s] * L[1], org[2] + tt[s] * L[2]};
            cell_of(g, q, cells[s], &cl[s]);
            dv[s] = tri_value(&cl[s], sdf) - bias;
            tt[s + 1] = tt[s] + (capped[s] ? (double)max_step : dv[s]);
        }
        const int i = argmin;
        const double d = dv[i], dp = i > 0 ? dv[i - 1] : INFINITY;
        const double y = i > 0 ? d * d / (2 * dp) : 0.0;
        const double e2 = d * d - y * y;
        const double e = e_pos32 && e2 > 0 ? sqrt(e2) : 0.0;
        const int den_tiny = den_tiny32;
        const double den = den_tiny ? 1e-6 : tt[i] - y;
        const double res = k * e / den;
        const double vis = res;
        loss += (vis - tg) * (vis - tg);
        if (!gsdf && !gl) continue;
        /* --- reverse mode along the frozen path */
        const double gr = 2 * (vis - tg);
        double gd[OR_MAX_STEPS], gt[OR_MAX_STEPS + 1];
        for (int s = 0; s <= i + 1; ++s) {
            gt[s] = 0;
            if (s <= i) gd[s] = 0;
        }
        const double ge = gr * k / den;
        double gy = 0;
        if (!den_tiny) {
            gt[i] += -gr * k * e / (den * den);
            gy += gr * k * e / (den * den);
        }
        if (e > 0) {
            gd[i] += ge * d / e;
            gy += ge * (-y / e);
        }
        if (i > 0) {
            gd[i] += gy * d / dp;
            gd[i - 1] += gy * (-d * d / (2 * dp * dp));
        }
        for (int s = i; s >= 0; --s) {
            if (s < i) {
                gt[s] += gt[s + 1];
                if (!capped[s]) gd[s] += gt[s + 1];
            }
            double w[8], grad[3];
            tri_weights(&cl[s], sdf, w, grad);
            if (gsdf)
                for (int b = 0; b < 8; ++b) gsdf[cl[s].c[b]] += gd[s] * w[b];
            const double gq[3] = {gd[s] * grad[0], gd[s] * grad[1], gd[s] * grad[2]};
            gt[s] += d_dot(gq, L);
            for (int a = 0; a < 3; ++a) gL[a] += gq[a] * tt[s];
        }
    }
    if (gl) {
        /* L = l / |l| */
        const double LgL = d_dot(L, gL);
        for (int a = 0; a < 3; ++a) gl[a] += (gL[a] - L[a] * LgL) / len;
    }
    return loss;
}
