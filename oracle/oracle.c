/*
 * CPU ORACLE for geometry-TSDF and asymmetric colour-volume integration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The CUDA path
 * shares no code with it.
 *
 * It is the plain definition, voxel by voxel, in the order the paper gives:
 *   Section IV.B, Eq. 5  voxel -> current depth camera   P_vc = R_n P_v + t_n
 *   Eq. 6 (Eq. 1)        projection with K_c, frustum test, depth fetch
 *   Eq. 7                back-projection of the depth pixel, sigma gate
 *   Eq. 2-4              depth camera -> HD camera -> HD pixel
 *   Eq. 9                running colour average (sample weight W = 1, so the
 *                        stored weight counts observing frames, capped)
 * plus the geometry (TSDF) update the paper inherits from KinectFusion
 * (Section III), and the trilinear TSDF band gate on colour voxels.  The
 * readings taken where the paper is silent are listed at each step.
 *
 * Arithmetic is IEEE binary32 in exactly the order written (compile with
 * -ffp-contract=off, no fast-math); fmaf() is the correctly rounded fused
 * multiply-add.  Integer decisions (pixel choice, gates, weights, colours) are
 * therefore taken in the same precision as in the CUDA kernels, which makes
 * weights and colours comparable bit for bit.  Frame constants (the inverse
 * pose and K_c^-1) are computed in binary64 and rounded once.
 *
 * Volumes are linear, x fastest: index (z * Ny + y) * Nx + x.  Colour voxels
 * are packed R | G<<8 | B<<16 | weight<<24.
 *
 * A z-slab of a larger volume (several devices or hosts each holding part of
 * one scan) is the same computation over a range of z: the parameters carry
 * the global z index of the slab's first geometry and colour voxel, every
 * voxel centre is taken at its global index, and the trilinear band gate
 * addresses the slab's geometry by global index minus that offset.  A slab
 * whose geometry extends one voxel beyond its colour range on each side
 * (where the volume continues) computes exactly the whole volume's values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t ng[3];        /* geometry dims (x, y, z) */
    int32_t nc[3];        /* colour dims (x, y, z) */
    float s_g;            /* geometry voxel size (m) */
    float s_c;            /* colour voxel size (m) */
    float origin[3];      /* world position of the volumes' minimum corner (m) */
    float mu;             /* truncation distance (m) */
    int32_t max_weight;   /* weight cap, 1..255 */
    float sigma;          /* depth-distance gate, Eq. 7 (m) */
    float band;           /* TSDF band gate, normalised units */
    int32_t colour_mode;  /* 0 = counting weight (Eq. 9 with W = 1); 1 = Eq. 8-10 */
    int32_t sample_mode;  /* 0 = nearest HD pixel; 1 = bilinear */
    int32_t update_free_space; /* 1: voxels with sdf > mu are updated with t = 1 */
    int32_t n_threads;    /* OpenMP threads for timing; 1 = reference mode */
    int32_t zoff_g;       /* z-slab of a larger volume: global z index of local geometry z = 0 */
    int32_t zoff_c;       /* and of local colour z = 0 (0, 0 for a whole volume) */
} orc_params;

typedef struct {
    float R[9], t[3];     /* (R_n, t_n): world -> current depth camera, Eq. 5 */
    float Kd[9], Kdi[9];  /* K_c and K_c^-1 */
    float Kr[9];          /* K_hd */
    float Rc[9], tc[3];   /* (R_calib, t_calib), Eq. 3 */
    float inv_mu, sigma2, inv_sg;
    int32_t dw, dh, cw, ch;
} orc_frame;

/* --------------------------------------------------- frame constants ---- */
/* T_world_depth maps depth-camera coordinates to world; Eq. 5 needs its
 * inverse.  R_n is the exact transpose; t_n = -(R^T t) in binary64, rounded
 * once.  K^-1 is the adjugate over the determinant, in binary64, rounded once. */
static void orc_frame_setup(orc_frame* f, const orc_params* p, const float Kd[9], const float Kr[9],
                            const float Twd[16], const float Tdr[16], int dw, int dh, int cw, int ch) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) f->R[r * 3 + c] = Twd[c * 4 + r];
    for (int i = 0; i < 3; ++i) {
        double s = (double)Twd[0 * 4 + i] * (double)Twd[0 * 4 + 3];
        s = s + (double)Twd[1 * 4 + i] * (double)Twd[1 * 4 + 3];
        s = s + (double)Twd[2 * 4 + i] * (double)Twd[2 * 4 + 3];
        f->t[i] = (float)(-s);
    }
    double a = Kd[0], b = Kd[1], c = Kd[2], d = Kd[3], e = Kd[4], ff = Kd[5], g = Kd[6], h = Kd[7], i = Kd[8];
    double A = e * i - ff * h, B = ff * g - d * i, C = d * h - e * g;
    double det = (a * A + b * B) + c * C;
    double adj[9] = {A, c * h - b * i, b * ff - c * e,
                     B, a * i - c * g, c * d - a * ff,
                     C, b * g - a * h, a * e - b * d};
    for (int k = 0; k < 9; ++k) f->Kdi[k] = (float)(adj[k] / det);
    memcpy(f->Kd, Kd, sizeof(float) * 9);
    memcpy(f->Kr, Kr, sizeof(float) * 9);
    for (int r = 0; r < 3; ++r) {
        for (int cc = 0; cc < 3; ++cc) f->Rc[r * 3 + cc] = Tdr[r * 4 + cc];
        f->tc[r] = Tdr[r * 4 + 3];
    }
    f->inv_mu = 1.0f / p->mu;
    f->sigma2 = p->sigma * p->sigma;
    f->inv_sg = 1.0f / p->s_g;
    f->dw = dw; f->dh = dh; f->cw = cw; f->ch = ch;
}

/* ------------------------------------------------------------ helpers --- */
/* Rigid motion y = R x + t (Eq. 3, Eq. 5), each row as fmaf chains. */
static void rigid(const float R[9], const float t[3], float x, float y, float z, float out[3]) {
    for (int r = 0; r < 3; ++r)
        out[r] = fmaf(R[r * 3 + 0], x, fmaf(R[r * 3 + 1], y, fmaf(R[r * 3 + 2], z, t[r])));
}

/* Eq. 1 / Eq. 6 / Eq. 4: (xh, yh, zh) = K (X, Y, Z); u = xh / zh, v = yh / zh
 * taken as one correctly rounded reciprocal and two products.  Points with
 * zh <= 0 are behind the camera (the frustum test of Section IV.B). */
static int project(const float K[9], float X, float Y, float Z, float* u, float* v) {
    float xh = fmaf(K[0], X, fmaf(K[1], Y, K[2] * Z));
    float yh = fmaf(K[3], X, fmaf(K[4], Y, K[5] * Z));
    float zh = fmaf(K[6], X, fmaf(K[7], Y, K[8] * Z));
    if (!(zh > 0.0f)) return 0;
    float rz = 1.0f / zh;
    *u = xh * rz;
    *v = yh * rz;
    return 1;
}

/* Nearest pixel (half-up rounding; the paper does not say) inside a W x H
 * image.  The bounds are tested in float before conversion, so NaN fails. */
static int nearest_pixel(float u, float v, int W, int H, int* iu, int* iv) {
    float fu = floorf(u + 0.5f), fv = floorf(v + 0.5f);
    if (!(fu >= 0.0f && fu <= (float)(W - 1) && fv >= 0.0f && fv <= (float)(H - 1))) return 0;
    *iu = (int)fu;
    *iv = (int)fv;
    return 1;
}

/* Voxel centre: origin + (index + 0.5) * voxel size (a reading: the paper
 * gives only integer voxel coordinates v). */
static float centre(float o, int i, float s) { return fmaf((float)i + 0.5f, s, o); }

static float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

/* -------------------------------------------------- geometry update ---- */
/* Projective TSDF update (KinectFusion, inherited in Section III; the paper
 * gives no formula, so this is the reading):
 *   D = depth at the voxel's pixel (0 = no measurement, skipped),
 *   sdf = D / 1000 - Z_c  (metres, along the optical axis),
 *   voxels with sdf < -mu are hidden and skipped,
 *   t = min(1, sdf / mu),
 *   F <- (F w + t) / (w + 1),  w <- min(w + 1, max_weight).
 * Averaging continues with w = max_weight once the cap is reached. */
/* One geometry voxel (x, y, z) whose F and w are at *Fv, *Wv; returns 1 if
 * it was updated. */
static int geo_voxel(const orc_params* p, const orc_frame* fr, float* Fv, uint8_t* Wv, const uint16_t* depth, int x,
                     int y, int z) {
    float P[3];
    rigid(fr->R, fr->t, centre(p->origin[0], x, p->s_g), centre(p->origin[1], y, p->s_g),
          centre(p->origin[2], z + p->zoff_g, p->s_g), P);
    float u, v;
    int iu, iv;
    if (!project(fr->Kd, P[0], P[1], P[2], &u, &v)) return 0;
    if (!nearest_pixel(u, v, fr->dw, fr->dh, &iu, &iv)) return 0;
    uint16_t D = depth[(size_t)iv * fr->dw + iu];
    if (D == 0) return 0;
    float d = (float)D * 0.001f;
    float sdf = d - P[2];
    if (sdf < -p->mu) return 0;
    if (!p->update_free_space && sdf > p->mu) return 0;
    float t = fminf(1.0f, sdf * fr->inv_mu);
    int w = *Wv;
    float wf = (float)w;
    *Fv = fmaf(*Fv, wf, t) / (wf + 1.0f);
    *Wv = (uint8_t)(w + 1 < p->max_weight ? w + 1 : p->max_weight);
    return 1;
}

static long long orc_geometry(const orc_params* p, const orc_frame* fr, float* F, uint8_t* W,
                              const uint16_t* depth) {
    const int nx = p->ng[0], ny = p->ng[1], nz = p->ng[2];
    long long updated = 0;
#pragma omp parallel for reduction(+ : updated) num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                size_t idx = ((size_t)z * ny + y) * nx + x;
                updated += geo_voxel(p, fr, &F[idx], &W[idx], depth, x, y, z);
            }
        }
    }
    return updated;
}

/* ---------------------------------------------------- colour update ---- */
/* Trilinear TSDF at grid coordinate g (geometry voxel units, centres at
 * integers).  Returns 0 when any of the 8 corners is outside the volume or
 * has weight 0 (never observed). */
/* Geometry voxel (x, y, z) as seen by the band gate: returns its weight
 * (0 = never observed) and its TSDF in *f. */
typedef int (*corner_fn)(const void* ctx, int x, int y, int z, float* f);

typedef struct {
    const orc_params* p;
    const float* F;
    const uint8_t* W;
} dense_geo;

static int dense_corner(const void* ctx, int x, int y, int z, float* f) {
    const dense_geo* d = (const dense_geo*)ctx;
    size_t idx = ((size_t)z * d->p->ng[1] + y) * d->p->ng[0] + x;
    *f = d->F[idx];
    return d->W[idx];
}

static int trilinear(const orc_params* p, corner_fn corner, const void* ctx, const float g[3], float* out) {
    float i0f[3], fr[3];
    int i0[3];
    for (int a = 0; a < 3; ++a) {
        i0f[a] = floorf(g[a]);
        fr[a] = g[a] - i0f[a];
        /* local cell of a z-slab: global index minus the slab's offset */
        const int lo = a == 2 ? p->zoff_g : 0;
        if (!(i0f[a] >= (float)lo && i0f[a] + 1.0f <= (float)(lo + p->ng[a] - 1))) return 0;
        i0[a] = (int)i0f[a] - lo;
    }
    float c[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                float f;
                if (corner(ctx, i0[0] + dx, i0[1] + dy, i0[2] + dz, &f) == 0) return 0;
                c[dz][dy][dx] = f;
            }
    /* lerp along x, then y, then z */
    float c00 = lerpf(c[0][0][0], c[0][0][1], fr[0]);
    float c10 = lerpf(c[0][1][0], c[0][1][1], fr[0]);
    float c01 = lerpf(c[1][0][0], c[1][0][1], fr[0]);
    float c11 = lerpf(c[1][1][0], c[1][1][1], fr[0]);
    float c0 = lerpf(c00, c10, fr[1]);
    float c1 = lerpf(c01, c11, fr[1]);
    *out = lerpf(c0, c1, fr[2]);
    return 1;
}

/* Bilinear cell of HD position (u, v): the upper-left pixel (floor u,
 * floor v) of the 2x2 footprint, which must lie inside the W x H image.
 * Returns 0 when it does not (tested in float, so NaN fails). */
static int bilinear_cell(float u, float v, int W, int H, float* x0, float* y0) {
    *x0 = floorf(u);
    *y0 = floorf(v);
    return *x0 >= 0.0f && *x0 + 1.0f <= (float)(W - 1) && *y0 >= 0.0f && *y0 + 1.0f <= (float)(H - 1);
}

/* HD pixel value HD(x_hd, y_hd) (Eq. 9): nearest pixel, or bilinear over the
 * 2x2 neighbourhood (which must lie inside the image), rounded half-up. */
static int sample_rgb(const orc_params* p, const orc_frame* fr, const uint8_t* rgb, float u, float v,
                      uint32_t s[3]) {
    if (p->sample_mode == 0) {
        int iu, iv;
        if (!nearest_pixel(u, v, fr->cw, fr->ch, &iu, &iv)) return 0;
        const uint8_t* px = rgb + ((size_t)iv * fr->cw + iu) * 3;
        for (int c = 0; c < 3; ++c) s[c] = px[c];
        return 1;
    }
    float x0, y0;
    if (!bilinear_cell(u, v, fr->cw, fr->ch, &x0, &y0)) return 0;
    float ax = u - x0, ay = v - y0;
    int ix = (int)x0, iy = (int)y0;
    const uint8_t* r0 = rgb + ((size_t)iy * fr->cw + ix) * 3;
    const uint8_t* r1 = r0 + (size_t)fr->cw * 3;
    for (int c = 0; c < 3; ++c) {
        float p00 = (float)r0[c], p10 = (float)r0[3 + c], p01 = (float)r1[c], p11 = (float)r1[3 + c];
        float top = fmaf(ax, p10 - p00, p00);
        float bot = fmaf(ax, p11 - p01, p01);
        float val = fmaf(ay, bot - top, top);
        s[c] = (uint32_t)floorf(val + 0.5f);
    }
    return 1;
}

/* Back-projection of depth pixel (iu, iv) with depth d (Eq. 7, read as
 * d * K_c^-1 (x, y, 1): the homogeneous form of Eq. 1/2). */
static void back_project(const orc_frame* fr, int iu, int iv, float d, float P[3]) {
    float fu = (float)iu, fv = (float)iv;
    for (int r = 0; r < 3; ++r) {
        float q = fmaf(fr->Kdi[r * 3 + 0], fu, fmaf(fr->Kdi[r * 3 + 1], fv, fr->Kdi[r * 3 + 2]));
        P[r] = d * q;
    }
}

/* Colour-volume update, run after the geometry update of the same frame.
 * For each colour voxel v (Section IV.B):
 *   Eq. 5      P_vc = R_n P_v + t_n
 *   Eq. 6      project with K_c; outside the frustum -> skip
 *              D = depth at that pixel; D == 0 -> skip
 *   Eq. 7      P_vd = back-projection of that pixel; |P_vc - P_vd| > sigma -> skip
 *   band gate  trilinear TSDF at P_v (post-update geometry) must exist and
 *              satisfy |F| <= band (the voxel lies near the fused surface)
 *   Eq. 3, 4   P_hd = R_calib P_vc + t_calib, project with K_hd; outside -> skip
 *   Eq. 9      counting mode: C <- (C w + HD + floor((w+1)/2)) div (w + 1)
 *              per 8-bit channel, w <- min(w + 1, max_weight).
 * colour_mode 1 (Eq. 8-10) is handled by orc_colour_paper_normal. */
static int orc_paper_normal_update(const orc_params* p, const orc_frame* fr, const uint16_t* depth,
                                   int iu, int iv, const float Pd[3], const float Pc[3],
                                   uint32_t* vox, const uint32_t s[3]);

/* The depth-side gates of colour voxel (x, y, z): Eq. 5, Eq. 6 (frustum and
 * D > 0), Eq. 7 (sigma) and the trilinear band gate.  On success returns 1
 * with the voxel in the current depth camera (Pc), its depth pixel and the
 * back-projected depth point (Pd). */
static int colour_depth_gates(const orc_params* p, const orc_frame* fr, corner_fn corner, const void* ctx,
                              const uint16_t* depth, int x, int y, int z, float Pc[3], int* iu, int* iv,
                              float Pd[3]) {
    float pw[3] = {centre(p->origin[0], x, p->s_c), centre(p->origin[1], y, p->s_c),
                   centre(p->origin[2], z + p->zoff_c, p->s_c)};
    rigid(fr->R, fr->t, pw[0], pw[1], pw[2], Pc);
    float u, v;
    if (!project(fr->Kd, Pc[0], Pc[1], Pc[2], &u, &v)) return 0;
    if (!nearest_pixel(u, v, fr->dw, fr->dh, iu, iv)) return 0;
    uint16_t D = depth[(size_t)(*iv) * fr->dw + *iu];
    if (D == 0) return 0;
    float d = (float)D * 0.001f;
    back_project(fr, *iu, *iv, d, Pd);
    float ex = Pc[0] - Pd[0], ey = Pc[1] - Pd[1], ez = Pc[2] - Pd[2];
    float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    if (dist2 > fr->sigma2) return 0;
    float g[3], Ft;
    for (int a = 0; a < 3; ++a) g[a] = fmaf(pw[a] - p->origin[a], fr->inv_sg, -0.5f);
    if (!trilinear(p, corner, ctx, g, &Ft)) return 0;
    if (!(fabsf(Ft) <= p->band)) return 0;
    return 1;
}

/* Eq. 3-4: the voxel's point P_vc in the depth camera, moved to the HD camera
 * (P_hd = R_calib P_vc + t_calib) and projected with K_hd.  Returns 0 behind
 * the HD camera. */
static int hd_position(const orc_frame* fr, const float Pc[3], float* uh, float* vh) {
    float Ph[3];
    rigid(fr->Rc, fr->tc, Pc[0], Pc[1], Pc[2], Ph);
    return project(fr->Kr, Ph[0], Ph[1], Ph[2], uh, vh);
}

/* One colour voxel (x, y, z) whose packed colour is at *Cv; the band gate
 * reads the geometry through `corner`.  Returns 1 if it was updated. */
static int colour_voxel(const orc_params* p, const orc_frame* fr, corner_fn corner, const void* ctx, uint32_t* Cv,
                        const uint16_t* depth, const uint8_t* rgb, int x, int y, int z) {
    float Pc[3], Pd[3];
    int iu, iv;
    if (!colour_depth_gates(p, fr, corner, ctx, depth, x, y, z, Pc, &iu, &iv, Pd)) return 0;
    float uh, vh;
    if (!hd_position(fr, Pc, &uh, &vh)) return 0;
    uint32_t s[3];
    if (!sample_rgb(p, fr, rgb, uh, vh, s)) return 0;
    if (p->colour_mode == 1) return orc_paper_normal_update(p, fr, depth, iu, iv, Pd, Pc, Cv, s);
    uint32_t cv = *Cv;
    uint32_t w = cv >> 24;
    uint32_t out = 0;
    for (int c = 0; c < 3; ++c) {
        uint32_t cc = (cv >> (8 * c)) & 0xFFu;
        uint32_t nc = (cc * w + s[c] + ((w + 1u) >> 1)) / (w + 1u);
        out |= nc << (8 * c);
    }
    uint32_t wn = w + 1u < (uint32_t)p->max_weight ? w + 1u : (uint32_t)p->max_weight;
    *Cv = out | (wn << 24);
    return 1;
}

static long long orc_colour(const orc_params* p, const orc_frame* fr, const float* F, const uint8_t* W,
                            uint32_t* C, const uint16_t* depth, const uint8_t* rgb) {
    const int nx = p->nc[0], ny = p->nc[1], nz = p->nc[2];
    const dense_geo geo = {p, F, W};
    long long updated = 0;
#pragma omp parallel for reduction(+ : updated) num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                size_t idx = ((size_t)z * ny + y) * nx + x;
                updated += colour_voxel(p, fr, dense_corner, &geo, &C[idx], depth, rgb, x, y, z);
            }
        }
    }
    return updated;
}

/* Eq. 8-10 colour weighting (colour_mode 1).
 *   Eq. 8: N = (P1 - P_vd) x (P2 - P_vd), P1/P2 the back-projections of the
 *          depth pixels one to the right and one below (both must be inside
 *          the image with non-zero depth; the paper is silent on borders).
 *   W = N^ . (P_vc / |P_vc|), the cosine between the normal and the viewing
 *       direction from the camera to the point; a surface facing the camera
 *       gives W > 0, and W <= 0 is skipped.
 *   W is stored as an 8-bit fixed-point value wq = floor(255 W + 1/2).
 *   Gate: W > 0.8 W_pre, in integers 5 wq > 4 w_pre.
 *   Eq. 9: C <- (C w_pre + HD wq + floor((w_pre + wq)/2)) div (w_pre + wq).
 *   Eq. 10: W_new = W_pre + W (1 - W_pre), in 1/255 fixed point:
 *           w_new = w_pre + (wq (255 - w_pre) + 127) div 255. */
static int orc_paper_normal_update(const orc_params* p, const orc_frame* fr, const uint16_t* depth,
                                   int iu, int iv, const float Pd[3], const float Pc[3],
                                   uint32_t* vox, const uint32_t s[3]) {
    (void)p;
    if (!(iu + 1 <= fr->dw - 1 && iv + 1 <= fr->dh - 1)) return 0;
    uint16_t D1 = depth[(size_t)iv * fr->dw + iu + 1];
    uint16_t D2 = depth[(size_t)(iv + 1) * fr->dw + iu];
    if (D1 == 0 || D2 == 0) return 0;
    float P1[3], P2[3];
    back_project(fr, iu + 1, iv, (float)D1 * 0.001f, P1);
    back_project(fr, iu, iv + 1, (float)D2 * 0.001f, P2);
    float a[3] = {P1[0] - Pd[0], P1[1] - Pd[1], P1[2] - Pd[2]};
    float b[3] = {P2[0] - Pd[0], P2[1] - Pd[1], P2[2] - Pd[2]};
    float n[3] = {fmaf(a[1], b[2], -(a[2] * b[1])), fmaf(a[2], b[0], -(a[0] * b[2])),
                  fmaf(a[0], b[1], -(a[1] * b[0]))};
    float nn = sqrtf(fmaf(n[0], n[0], fmaf(n[1], n[1], n[2] * n[2])));
    float pn = sqrtf(fmaf(Pc[0], Pc[0], fmaf(Pc[1], Pc[1], Pc[2] * Pc[2])));
    if (!(nn > 0.0f && pn > 0.0f)) return 0;
    /* with x right, y down, z forward, (right) x (down) points along the
     * viewing direction for a surface facing the camera, so N.P_vc > 0 there */
    float dot = fmaf(n[0], Pc[0], fmaf(n[1], Pc[1], n[2] * Pc[2]));
    float Wc = dot / (nn * pn);
    if (!(Wc > 0.0f)) return 0;
    uint32_t wq = (uint32_t)floorf(fmaf(Wc, 255.0f, 0.5f));
    if (wq > 255u) wq = 255u;
    uint32_t cv = *vox;
    uint32_t wp = cv >> 24;
    if (!(5u * wq > 4u * wp)) return 0;
    uint32_t den = wp + wq;
    uint32_t out = 0;
    for (int c = 0; c < 3; ++c) {
        uint32_t cc = (cv >> (8 * c)) & 0xFFu;
        uint32_t nc = (cc * wp + s[c] * wq + (den >> 1)) / den;
        out |= nc << (8 * c);
    }
    uint32_t wn = wp + (wq * (255u - wp) + 127u) / 255u;
    *vox = out | (wn << 24);
    return 1;
}

/* ------------------------------------------------------------- public --- */
/* Integrate one frame: the geometry update over the whole geometry volume,
 * then the colour update over the whole colour volume (which reads the
 * updated geometry).  depth: uint16 mm (dh x dw); rgb: uint8 HWC (ch x cw x 3);
 * K row-major 3x3; T row-major 4x4.  counts (nullable) receives the number of
 * updated geometry and colour voxels.  Returns 0. */
int orc_integrate(const orc_params* p, float* F, uint8_t* W, uint32_t* C, const uint16_t* depth, int dw,
                  int dh, const uint8_t* rgb, int cw, int ch, const float Kd[9], const float Kr[9],
                  const float Twd[16], const float Tdr[16], long long counts[2]) {
    orc_frame fr;
    orc_frame_setup(&fr, p, Kd, Kr, Twd, Tdr, dw, dh, cw, ch);
    long long g = orc_geometry(p, &fr, F, W, depth);
    long long c = orc_colour(p, &fr, F, W, C, depth, rgb);
    if (counts) { counts[0] = g; counts[1] = c; }
    return 0;
}

/* Geometry update only (for tests of the TSDF step on its own). */
long long orc_integrate_geometry(const orc_params* p, float* F, uint8_t* W, const uint16_t* depth, int dw,
                                 int dh, const float Kd[9], const float Twd[16]) {
    orc_frame fr;
    float I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    orc_frame_setup(&fr, p, Kd, Kd, Twd, I, dw, dh, dw, dh);
    return orc_geometry(p, &fr, F, W, depth);
}

/* The frame constants, for inspection by tests. */
void orc_frame_constants(const orc_params* p, const float Kd[9], const float Kr[9], const float Twd[16],
                         const float Tdr[16], float R[9], float t[3], float Kdi[9]) {
    orc_frame fr;
    orc_frame_setup(&fr, p, Kd, Kr, Twd, Tdr, 1, 1, 1, 1);
    memcpy(R, fr.R, sizeof fr.R);
    memcpy(t, fr.t, sizeof fr.t);
    memcpy(Kdi, fr.Kdi, sizeof fr.Kdi);
}

int orc_params_size(void) { return (int)sizeof(orc_params); }

/* Geometry update of one frame, then the list of colour voxels that pass the
 * depth-side gates (colour_depth_gates) against the updated geometry: the
 * set S_k of the photometric loss.  Writes at most cap linear colour indices
 * (ascending) to out and returns how many pass. */
long long orc_record_gates(const orc_params* p, float* F, uint8_t* W, const uint16_t* depth, int dw, int dh,
                           const float Kd[9], const float Twd[16], uint32_t* out, long long cap) {
    orc_frame fr;
    float I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    orc_frame_setup(&fr, p, Kd, Kd, Twd, I, dw, dh, dw, dh);
    orc_geometry(p, &fr, F, W, depth);
    const int nx = p->nc[0], ny = p->nc[1], nz = p->nc[2];
    const dense_geo geo = {p, F, W};
    /* the gates of every voxel (in parallel for timing runs), then the list in
     * ascending order */
    uint8_t* pass = (uint8_t*)malloc((size_t)nx * ny * nz);
    if (!pass) return -1;
#pragma omp parallel for num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                float Pc[3], Pd[3];
                int iu, iv;
                pass[((size_t)z * ny + y) * nx + x] =
                    (uint8_t)colour_depth_gates(p, &fr, dense_corner, &geo, depth, x, y, z, Pc, &iu, &iv, Pd);
            }
    long long n = 0;
    for (size_t i = 0; i < (size_t)nx * ny * nz; ++i)
        if (pass[i]) {
            if (n < cap) out[n] = (uint32_t)i;
            ++n;
        }
    free(pass);
    return n;
}

/* Bilinear HD cells of the photometric loss (the integer decision of each
 * sample): for every (frame k, colour voxel) pair, the voxel centre moved by
 * frame k's depth-camera motion (R_n, t_n) (Eq. 5), then by the depth-to-HD
 * extrinsic T (Eq. 3) and projected with K_hd (Eq. 4) -- the steps of the
 * colour update above (hd_position) -- and the 2x2 footprint test of the
 * bilinear sampling (bilinear_cell).  cells[2 i], cells[2 i + 1] = (x0, y0)
 * of pair i, or INT32_MIN twice when the sample is behind the camera or its
 * footprint leaves the cw x ch image.
 *   nc, s_c, origin   the colour grid;  Rn, tn  n_frames x 9 / x 3
 *   offsets, idx      pairs of frame k are idx[offsets[k] .. offsets[k+1])
 *   Kr, Tdr           row-major 3x3 K_hd and 4x4 T_depth_rgb (binary32) */
void orc_hd_cells(const int32_t nc[3], float s_c, const float origin[3], int n_frames, const float* Rn,
                  const float* tn, const int64_t* offsets, const uint32_t* idx, const float Kr[9], const float Tdr[16],
                  int cw, int ch, int32_t* cells) {
    orc_frame fr;
    memset(&fr, 0, sizeof fr);
    memcpy(fr.Kr, Kr, sizeof fr.Kr);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) fr.Rc[r * 3 + c] = Tdr[r * 4 + c];
        fr.tc[r] = Tdr[r * 4 + 3];
    }
    fr.cw = cw;
    fr.ch = ch;
    const uint32_t nx = (uint32_t)nc[0], ny = (uint32_t)nc[1];
    for (int k = 0; k < n_frames; ++k) {
        memcpy(fr.R, Rn + 9 * k, sizeof fr.R);
        memcpy(fr.t, tn + 3 * k, sizeof fr.t);
        for (int64_t i = offsets[k]; i < offsets[k + 1]; ++i) {
            const uint32_t v = idx[i];
            const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / (nx * ny));
            float Pc[3], uh, vh, x0, y0;
            rigid(fr.R, fr.t, centre(origin[0], x, s_c), centre(origin[1], y, s_c), centre(origin[2], z, s_c), Pc);
            int32_t cx = INT32_MIN, cy = INT32_MIN;
            if (hd_position(&fr, Pc, &uh, &vh) && bilinear_cell(uh, vh, cw, ch, &x0, &y0)) {
                cx = (int32_t)x0;
                cy = (int32_t)y0;
            }
            cells[2 * i] = cx;
            cells[2 * i + 1] = cy;
        }
    }
}

/* ---------------------------------------------------------- sampled ---- */
/* Sampled replay of one frame, for parity checks at sizes where the whole
 * volumes are too large for the oracle: the same per-voxel updates as
 * orc_integrate, applied to a list of geometry voxels (linear indices,
 * ascending, with their F and w) and then to a list of colour voxels (with
 * their packed colours).  The band gate of a colour voxel reads its trilinear
 * corners from the geometry list; a corner missing from the list is counted
 * in *missing and read as unobserved.  Returns 0. */
typedef struct {
    const orc_params* p;
    const uint64_t* lin;
    const float* F;
    const uint8_t* W;
    int64_t n;
    long long* missing;
} sparse_geo;

static int sparse_corner(const void* ctx, int x, int y, int z, float* f) {
    const sparse_geo* s = (const sparse_geo*)ctx;
    uint64_t key = ((uint64_t)z * (uint64_t)s->p->ng[1] + (uint64_t)y) * (uint64_t)s->p->ng[0] + (uint64_t)x;
    int64_t lo = 0, hi = s->n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (s->lin[mid] == key) {
            *f = s->F[mid];
            return s->W[mid];
        }
        if (s->lin[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    #pragma omp atomic
    (*s->missing)++;
    *f = 0.0f;
    return 0;
}

int orc_sparse_frame(const orc_params* p, const uint16_t* depth, int dw, int dh, const uint8_t* rgb, int cw, int ch,
                     const float Kd[9], const float Kr[9], const float Twd[16], const float Tdr[16], int64_t ng,
                     const uint64_t* g_lin, float* gF, uint8_t* gW, int64_t nc, const uint64_t* c_lin, uint32_t* cC,
                     long long* missing) {
    orc_frame fr;
    orc_frame_setup(&fr, p, Kd, Kr, Twd, Tdr, dw, dh, cw, ch);
    const uint64_t gx = (uint64_t)p->ng[0], gy = (uint64_t)p->ng[1];
    const uint64_t cx = (uint64_t)p->nc[0], cy = (uint64_t)p->nc[1];
#pragma omp parallel for num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 256)
    for (int64_t i = 0; i < ng; ++i) {
        uint64_t l = g_lin[i];
        geo_voxel(p, &fr, &gF[i], &gW[i], depth, (int)(l % gx), (int)((l / gx) % gy), (int)(l / (gx * gy)));
    }
    sparse_geo geo = {p, g_lin, gF, gW, ng, missing};
#pragma omp parallel for num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 256)
    for (int64_t i = 0; i < nc; ++i) {
        uint64_t l = c_lin[i];
        colour_voxel(p, &fr, sparse_corner, &geo, &cC[i], depth, rgb, (int)(l % cx), (int)((l / cx) % cy),
                     (int)(l / (cx * cy)));
    }
    return 0;
}
