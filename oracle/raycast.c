/*
 * CPU ORACLE of the ray caster of the fused volumes: the paper shows the
 * scan to the user by ray casting both volumes (abstract) and tracks the
 * camera against a surface vertex map predicted by ray tracing the geometry
 * volume (Section III).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests and the smoke check may load this
 * file's library.  The CUDA path shares no code with it.
 *
 * Definition, binary32 with the operation order written here (compiled with
 * -ffp-contract=off; fmaf is the correctly rounded fused multiply-add):
 *
 *   ray of pixel (x, y):  dc = K^-1 (x, y, 1) (rows summed as fmaf(k0, x,
 *     fmaf(k1, y, k2)); K^-1 binary64 rounded once), nd = 1 / sqrtf(dc . dc),
 *     d = (R dc) * nd (R = rotation of T_world_camera, rows as fmaf(r0, dcx,
 *     fmaf(r1, dcy, r2 * dcz))), o = translation of T_world_camera; a point of
 *     the ray is p(t) = fmaf(t, d, o) per axis, t the distance from o.
 *   TSDF at p: the trilinear interpolation of the colour band gate
 *     (g = fmaf(p - origin, 1/s_g, -1/2), i0 = floor(g), f = g - i0, lerp
 *     along x, then y, then z); it exists only when all eight corners lie in
 *     the volume and are observed (w > 0).
 *   march: t = near; at each sample the TSDF F(t) is taken; the first sample
 *     with F <= 0 whose predecessor (the sample just before) had F > 0 ends
 *     the march with a hit; the next t is t + (F exists and F < 1 ? step_near
 *     : step_far), the fine step only inside the truncation band; the march
 *     stops without a hit once t > far.
 *   hit: t* = fmaf(t - t_prev, F_prev / (F_prev - F), t_prev) (linear
 *     interpolation of the zero crossing), vertex v = p(t*).
 *   normal: n_a = F(v + s_g e_a) - F(v - s_g e_a) (central differences of the
 *     trilinear TSDF; the shifted point changes only coordinate a, by one add
 *     or subtract); all six must exist and |n|^2 = fmaf(nx, nx, fmaf(ny, ny,
 *     nz * nz)) > 0, then n_a / sqrtf(|n|^2); else the normal is (0, 0, 0).
 *     It points from the inside (F < 0) to free space, toward the camera.
 *   colour: the colour voxel k_a = floorf((v_a - origin_a) * (1/s_c)) (1/s_c
 *     binary64 rounded once) when it lies in the colour volume; else 0.
 * Misses leave range 0, vertex and normal (0, 0, 0) and colour 0.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

typedef struct {
    int32_t ng[3], nc[3];
    float s_g, s_c;
    float origin[3];
    const float* F;      /* linear, x fastest */
    const uint8_t* W;
    const uint32_t* C;   /* packed RGBW, may be NULL */
} orc_rc_volume;

typedef struct {
    int32_t width, height;
    float Kinv[9];       /* binary64 inverse of K rounded once */
    float R[9], t[3];    /* camera -> world */
    float near_, far_, step_far, step_near;
    float inv_sg, inv_sc;
} orc_rc_camera;

static float rc_lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

/* Trilinear TSDF at world point p; returns 0 when a corner is outside the
 * volume or unobserved. */
static int rc_tsdf(const orc_rc_volume* v, const orc_rc_camera* c, const float p[3], float* out) {
    float g[3], fr[3];
    int i0[3];
    for (int a = 0; a < 3; ++a) {
        g[a] = fmaf(p[a] - v->origin[a], c->inv_sg, -0.5f);
        float fl = floorf(g[a]);
        if (!(fl >= 0.0f) || !(fl + 1.0f <= (float)(v->ng[a] - 1))) return 0;
        i0[a] = (int)fl;
        fr[a] = g[a] - fl;
    }
    float q[8];
    for (int k = 0; k < 8; ++k) {
        int x = i0[0] + (k & 1), y = i0[1] + ((k >> 1) & 1), z = i0[2] + (k >> 2);
        size_t idx = ((size_t)z * v->ng[1] + y) * v->ng[0] + x;
        if (v->W[idx] == 0) return 0;
        q[k] = v->F[idx];
    }
    float c00 = rc_lerp(q[0], q[1], fr[0]), c10 = rc_lerp(q[2], q[3], fr[0]);
    float c01 = rc_lerp(q[4], q[5], fr[0]), c11 = rc_lerp(q[6], q[7], fr[0]);
    float c0 = rc_lerp(c00, c10, fr[1]), c1 = rc_lerp(c01, c11, fr[1]);
    *out = rc_lerp(c0, c1, fr[2]);
    return 1;
}

static void rc_point(float t, const float d[3], const float o[3], float p[3]) {
    for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
}

/* One pixel.  Returns 1 on a hit. */
static int rc_pixel(const orc_rc_volume* v, const orc_rc_camera* c, int x, int y, float* range, float vert[3],
                    float nrm[3], uint32_t* rgbw) {
    const float fx = (float)x, fy = (float)y;
    const float* K = c->Kinv;
    float dc[3] = {fmaf(K[0], fx, fmaf(K[1], fy, K[2])), fmaf(K[3], fx, fmaf(K[4], fy, K[5])),
                   fmaf(K[6], fx, fmaf(K[7], fy, K[8]))};
    float nd = 1.0f / sqrtf(fmaf(dc[0], dc[0], fmaf(dc[1], dc[1], dc[2] * dc[2])));
    float d[3];
    for (int a = 0; a < 3; ++a)
        d[a] = fmaf(c->R[3 * a], dc[0], fmaf(c->R[3 * a + 1], dc[1], c->R[3 * a + 2] * dc[2])) * nd;
    *range = 0.0f;
    vert[0] = vert[1] = vert[2] = 0.0f;
    nrm[0] = nrm[1] = nrm[2] = 0.0f;
    *rgbw = 0u;
    float t = c->near_, tp = 0.0f, Fp = 0.0f;
    int has_prev = 0;
    while (t <= c->far_) {
        float p[3], F;
        rc_point(t, d, c->t, p);
        int ok = rc_tsdf(v, c, p, &F);
        if (ok && has_prev && Fp > 0.0f && F <= 0.0f) {
            float ts = fmaf(t - tp, Fp / (Fp - F), tp);
            rc_point(ts, d, c->t, vert);
            *range = ts;
            float n[3];
            int good = 1;
            for (int a = 0; a < 3 && good; ++a) {
                float pp[3] = {vert[0], vert[1], vert[2]}, pm[3] = {vert[0], vert[1], vert[2]};
                pp[a] = vert[a] + v->s_g;
                pm[a] = vert[a] - v->s_g;
                float fp, fm;
                good = rc_tsdf(v, c, pp, &fp) && rc_tsdf(v, c, pm, &fm);
                if (good) n[a] = fp - fm;
            }
            if (good) {
                float l2 = fmaf(n[0], n[0], fmaf(n[1], n[1], n[2] * n[2]));
                if (l2 > 0.0f) {
                    float l = sqrtf(l2);
                    for (int a = 0; a < 3; ++a) nrm[a] = n[a] / l;
                }
            }
            if (v->C) {
                int k[3], in = 1;
                for (int a = 0; a < 3; ++a) {
                    float q = floorf((vert[a] - v->origin[a]) * c->inv_sc);
                    in = in && q >= 0.0f && q < (float)v->nc[a];
                    k[a] = in ? (int)q : 0;
                }
                if (in) *rgbw = v->C[((size_t)k[2] * v->nc[1] + k[1]) * v->nc[0] + k[0]];
            }
            return 1;
        }
        has_prev = ok;
        if (ok) { Fp = F; tp = t; }
        t = t + ((ok && F < 1.0f) ? c->step_near : c->step_far);
    }
    return 0;
}

/* Ray-cast every pixel; outputs are height x width (x 3), any may be NULL.
 * Returns the number of hits. */
long long orc_raycast(const orc_rc_volume* v, const orc_rc_camera* c, float* range, float* vertex, float* normal,
                      uint32_t* rgbw) {
    long long hits = 0;
#pragma omp parallel for reduction(+ : hits) schedule(dynamic, 4)
    for (int y = 0; y < c->height; ++y) {
        for (int x = 0; x < c->width; ++x) {
            size_t i = (size_t)y * c->width + x;
            float r, vt[3], n[3];
            uint32_t col;
            hits += rc_pixel(v, c, x, y, &r, vt, n, &col);
            if (range) range[i] = r;
            if (vertex) for (int a = 0; a < 3; ++a) vertex[3 * i + a] = vt[a];
            if (normal) for (int a = 0; a < 3; ++a) normal[3 * i + a] = n[a];
            if (rgbw) rgbw[i] = col;
        }
    }
    return hits;
}

int orc_rc_sizes(int which) { return which == 0 ? (int)sizeof(orc_rc_volume) : (int)sizeof(orc_rc_camera); }
