/*
 * Seeded synthetic RGB-D sensor: ray-traced analytic scenes.
 *
 * This module stands in for the paper's captured scans (a Kinect depth camera
 * rigidly paired with an HD RGB camera, Section IV.A / Section V).  It renders
 * what such a rig would see of a scene made of planes, axis-aligned boxes and
 * spheres with procedural albedo.  It holds none of the fusion method's
 * arithmetic: it only produces input images.  Both the CPU oracle and the CUDA
 * path are fed from it.
 *
 * Conventions: world z is up; cameras look along +z with x right and y down;
 * a pose T_world_cam maps camera coordinates to world coordinates (row-major
 * 4x4).  Pixel (i, j) has its centre at image coordinates (i, j).
 *
 * Randomness (depth noise, dropout) comes from splitmix64 keyed on
 * (seed, frame, pixel), so a frame's bytes depend only on its inputs, not on
 * thread count or rendering order.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

enum { PRIM_PLANE = 0, PRIM_BOX = 1, PRIM_SPHERE = 2 };
enum { ALB_CHECKER = 0, ALB_NOISE = 1, ALB_CONSTANT = 2 };

/* One primitive.  Plane: horizontal plane z = c[2].  Box: centre c, half
 * extents e.  Sphere: centre c, radius e[0]. */
typedef struct {
    int32_t kind;
    int32_t albedo;
    double c[3];
    double e[3];
    double col_a[3]; /* albedo colour A (0..255) */
    double col_b[3]; /* albedo colour B (0..255) */
    double scale;    /* checker cell size (m) or base noise frequency (1/m) */
    uint64_t seed;   /* noise lattice seed */
} synth_prim;

/* ---------------------------------------------------------------- RNG -- */
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}
static double u01(uint64_t h) { /* (0, 1) */
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static uint64_t pixel_key(uint64_t seed, uint64_t frame, uint64_t pix) {
    return splitmix64(splitmix64(splitmix64(seed) ^ (frame * 0xD1B54A32D192ED03ULL)) ^ pix);
}

/* ------------------------------------------------------- intersection -- */
/* Ray o + s d, s > 0.  Returns the nearest s or INFINITY. */
static double hit_plane(const synth_prim* p, const double o[3], const double d[3]) {
    if (d[2] == 0.0) return INFINITY;
    double s = (p->c[2] - o[2]) / d[2];
    return s > 1e-9 ? s : INFINITY;
}
static double hit_sphere(const synth_prim* p, const double o[3], const double d[3]) {
    double oc[3] = {o[0] - p->c[0], o[1] - p->c[1], o[2] - p->c[2]};
    double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - p->e[0] * p->e[0];
    double disc = b * b - a * c;
    if (disc < 0.0) return INFINITY;
    double sq = sqrt(disc);
    double s0 = (-b - sq) / a, s1 = (-b + sq) / a;
    if (s0 > 1e-9) return s0;
    if (s1 > 1e-9) return s1;
    return INFINITY;
}
static double hit_box(const synth_prim* p, const double o[3], const double d[3]) {
    double tmin = -INFINITY, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = p->c[a] - p->e[a], hi = p->c[a] + p->e[a];
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return INFINITY;
            continue;
        }
        double t0 = (lo - o[a]) / d[a], t1 = (hi - o[a]) / d[a];
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > tmin) tmin = t0;
        if (t1 < tmax) tmax = t1;
        if (tmin > tmax) return INFINITY;
    }
    if (tmin > 1e-9) return tmin;
    if (tmax > 1e-9) return tmax;
    return INFINITY;
}
static double hit_prim(const synth_prim* p, const double o[3], const double d[3]) {
    switch (p->kind) {
        case PRIM_PLANE: return hit_plane(p, o, d);
        case PRIM_BOX: return hit_box(p, o, d);
        case PRIM_SPHERE: return hit_sphere(p, o, d);
    }
    return INFINITY;
}
static int trace(const synth_prim* prims, int n, const double o[3], const double d[3], double* s_out) {
    int best = -1;
    double bs = INFINITY;
    for (int i = 0; i < n; ++i) {
        double s = hit_prim(&prims[i], o, d);
        if (s < bs) { bs = s; best = i; }
    }
    *s_out = bs;
    return best;
}

/* ------------------------------------------------------------ albedo -- */
static double lattice(uint64_t seed, int64_t x, int64_t y, int64_t z) {
    uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)x * 0x8CB92BA72F3D8DD7ULL ^
                                              splitmix64((uint64_t)y * 0xABC98388FB8FAC03ULL ^
                                                         (uint64_t)z * 0x9E3779B97F4A7C15ULL)));
    return u01(h);
}
static double smooth(double t) { return t * t * (3.0 - 2.0 * t); }
static double value_noise(uint64_t seed, double x, double y, double z) {
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
    double tx = smooth(x - fx), ty = smooth(y - fy), tz = smooth(z - fz);
    double v[2][2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) v[a][b][c] = lattice(seed, ix + a, iy + b, iz + c);
    double x00 = v[0][0][0] + tx * (v[1][0][0] - v[0][0][0]);
    double x10 = v[0][1][0] + tx * (v[1][1][0] - v[0][1][0]);
    double x01 = v[0][0][1] + tx * (v[1][0][1] - v[0][0][1]);
    double x11 = v[0][1][1] + tx * (v[1][1][1] - v[0][1][1]);
    double y0 = x00 + ty * (x10 - x00), y1 = x01 + ty * (x11 - x01);
    return y0 + tz * (y1 - y0);
}
static void albedo(const synth_prim* p, const double x[3], double rgb[3]) {
    double t = 0.0;
    switch (p->albedo) {
        case ALB_CHECKER: {
            double s = p->scale;
            /* offset by a quarter cell so faces at round coordinates do not flicker */
            int64_t k = (int64_t)floor(x[0] / s + 0.25) + (int64_t)floor(x[1] / s + 0.25) +
                        (int64_t)floor(x[2] / s + 0.25);
            t = (k & 1) ? 1.0 : 0.0;
            break;
        }
        case ALB_NOISE: {
            double f = p->scale, amp = 0.5, sum = 0.0, norm = 0.0;
            for (int o = 0; o < 3; ++o) {
                sum += amp * value_noise(p->seed + (uint64_t)o, x[0] * f, x[1] * f, x[2] * f);
                norm += amp;
                amp *= 0.5;
                f *= 2.0;
            }
            t = sum / norm;
            break;
        }
        case ALB_CONSTANT: t = 0.0; break;
        default: t = 0.0; break;
    }
    for (int c = 0; c < 3; ++c) rgb[c] = p->col_a[c] + t * (p->col_b[c] - p->col_a[c]);
}

/* ------------------------------------------------------------ camera -- */
typedef struct {
    double kinv[9];
    double R[9];
    double t[3];
} cam_t;

static void cam_setup(cam_t* c, const double K[9], const double T[16]) {
    /* inverse of a 3x3 via the adjugate */
    double a = K[0], b = K[1], cc = K[2], d = K[3], e = K[4], f = K[5], g = K[6], h = K[7], i = K[8];
    double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
    double det = a * A + b * B + cc * C;
    double inv[9] = {A, -(b * i - cc * h), b * f - cc * e,
                     B, a * i - cc * g, -(a * f - cc * d),
                     C, -(a * h - b * g), a * e - b * d};
    for (int k = 0; k < 9; ++k) c->kinv[k] = inv[k] / det;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c->R[r * 3 + k] = T[r * 4 + k];
        c->t[r] = T[r * 4 + 3];
    }
}
/* world-space ray through pixel centre (u, v); direction has camera-z = 1 */
static void cam_ray(const cam_t* c, double u, double v, double o[3], double d[3]) {
    double dc[3];
    for (int r = 0; r < 3; ++r) dc[r] = c->kinv[r * 3 + 0] * u + c->kinv[r * 3 + 1] * v + c->kinv[r * 3 + 2];
    /* normalise so that the camera-frame z component is exactly the depth parameter */
    double zc = dc[2];
    for (int r = 0; r < 3; ++r) dc[r] /= zc;
    for (int r = 0; r < 3; ++r) {
        d[r] = c->R[r * 3 + 0] * dc[0] + c->R[r * 3 + 1] * dc[1] + c->R[r * 3 + 2] * dc[2];
        o[r] = c->t[r];
    }
}

/* -------------------------------------------------------------- API -- */

/* Depth image (uint16 millimetres, 0 = invalid) of the camera with intrinsics
 * K (row-major 3x3) and pose T_world_cam.  noise_coeff: Kinect-like axial
 * noise sigma = noise_coeff * z^2 metres (0 disables); dropout: probability of
 * a 0 pixel; max_range: hits beyond it read 0. */
void synth_render_depth(const synth_prim* prims, int n, const double K[9], const double T[16],
                        int W, int H, uint64_t seed, uint64_t frame, double noise_coeff,
                        double dropout, double max_range, uint16_t* out) {
    cam_t cam;
    cam_setup(&cam, K, T);
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            double o[3], d[3], s;
            cam_ray(&cam, (double)i, (double)j, o, d);
            int hit = trace(prims, n, o, d, &s);
            uint16_t D = 0;
            if (hit >= 0 && s <= max_range) {
                uint64_t key = pixel_key(seed, frame, (uint64_t)j * (uint64_t)W + (uint64_t)i);
                double z = s;
                if (noise_coeff > 0.0) {
                    double u1 = u01(splitmix64(key ^ 1)), u2 = u01(splitmix64(key ^ 2));
                    double gauss = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                    z += noise_coeff * s * s * gauss;
                }
                double mm = floor(z * 1000.0 + 0.5);
                int drop = dropout > 0.0 && u01(splitmix64(key ^ 3)) < dropout;
                if (!drop && mm >= 1.0 && mm <= 65535.0 && z <= max_range) D = (uint16_t)mm;
            }
            out[(size_t)j * W + i] = D;
        }
    }
}

/* Unlit RGB image (uint8 HWC, R first) of the camera with intrinsics K and
 * pose T_world_cam.  Rays that miss every primitive read `background`. */
void synth_render_rgb(const synth_prim* prims, int n, const double K[9], const double T[16],
                      int W, int H, const double background[3], uint8_t* out) {
    cam_t cam;
    cam_setup(&cam, K, T);
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            double o[3], d[3], s, rgb[3];
            cam_ray(&cam, (double)i, (double)j, o, d);
            int hit = trace(prims, n, o, d, &s);
            if (hit >= 0) {
                double x[3] = {o[0] + s * d[0], o[1] + s * d[1], o[2] + s * d[2]};
                albedo(&prims[hit], x, rgb);
            } else {
                rgb[0] = background[0]; rgb[1] = background[1]; rgb[2] = background[2];
            }
            uint8_t* px = out + ((size_t)j * W + i) * 3;
            for (int c = 0; c < 3; ++c) {
                double v = floor(rgb[c] + 0.5);
                px[c] = (uint8_t)(v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v));
            }
        }
    }
}

/* Size of the primitive record, so the Python side can check its layout. */
int synth_prim_size(void) { return (int)sizeof(synth_prim); }
