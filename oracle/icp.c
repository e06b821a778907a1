/*
 * CPU ORACLE of camera tracking: the KinectFusion loop the paper builds on
 * (Section III).  A vertex map and normal map pyramid is computed from the
 * input depth map, and the camera motion is estimated by iterative closest
 * point against a predicted surface vertex map ray-traced from the geometry
 * volume (the prediction comes from raycast.c).  The paper gives no further
 * detail; the readings taken here (projective association, point-to-plane
 * error, gates, pyramid averaging, iteration counts) are stated at each step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests may load this file's library.
 * The CUDA path shares no code with it.
 *
 * Per-pixel geometry is binary32 in the operation order written here
 * (-ffp-contract=off; fmaf is the correctly rounded fused multiply-add), so
 * the integer decisions (which pixels correspond) can be compared exactly.
 * The normal equations are accumulated in binary64 from the binary32 terms,
 * solved in binary64, and the pose is kept in binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------- pyramid -- */
/* Level 0: depth in metres d = D * 0.001 (D = 0: no depth, 0).  Level l + 1,
 * pixel (x, y), from the 2 x 2 block (2x + i, 2y + j) of level l taken in the
 * order (0,0), (1,0), (0,1), (1,1): the mean of the block's valid depths that
 * lie within 0.03 m of its first valid depth (a reading: a plain average that
 * does not mix the two sides of a depth edge), summed in that order and
 * divided once; 0 when the block has no valid depth.  Level l is W >> l by
 * H >> l.  out holds the levels one after another. */
void orc_icp_pyramid(const uint16_t* depth, int W, int H, int levels, float* out) {
    for (int i = 0; i < W * H; ++i) out[i] = depth[i] ? (float)depth[i] * 0.001f : 0.0f;
    const float* prev = out;
    float* cur = out + (size_t)W * H;
    int w = W, h = H;
    for (int l = 1; l < levels; ++l) {
        const int w2 = w / 2, h2 = h / 2;
        for (int y = 0; y < h2; ++y)
            for (int x = 0; x < w2; ++x) {
                float first = 0.0f, sum = 0.0f;
                int n = 0;
                for (int k = 0; k < 4; ++k) {
                    const float d = prev[(size_t)(2 * y + (k >> 1)) * w + 2 * x + (k & 1)];
                    if (d == 0.0f) continue;
                    if (n == 0) first = d;
                    if (fabsf(d - first) <= 0.03f) {
                        sum = sum + d;
                        ++n;
                    }
                }
                cur[(size_t)y * w2 + x] = n ? sum / (float)n : 0.0f;
            }
        prev = cur;
        cur += (size_t)w2 * h2;
        w = w2;
        h = h2;
    }
}

/* Intrinsics of level l (a reading consistent with the block averaging: the
 * centre of block pixel (x, y) is level-0 pixel 2^l (x + 1/2) - 1/2):
 * f_l = f / 2^l, c_l = (c + 1/2) / 2^l - 1/2, in binary64 rounded once. */
void orc_icp_level_K(const float K[9], int l, float Kl[9]) {
    const double s = ldexp(1.0, -l);
    memset(Kl, 0, 9 * sizeof(float));
    Kl[0] = (float)((double)K[0] * s);
    Kl[4] = (float)((double)K[4] * s);
    Kl[2] = (float)(((double)K[2] + 0.5) * s - 0.5);
    Kl[5] = (float)(((double)K[5] + 0.5) * s - 0.5);
    Kl[8] = 1.0f;
}

/* ------------------------------------------------- vertex and normal maps -- */
/* Vertex V(x, y) = d K^-1 (x, y, 1) with K^-1 of a pinhole K in binary64
 * rounded once: X = d fmaf(1/fx, x, -cx/fx), Y = d fmaf(1/fy, y, -cy/fy),
 * Z = d (the back-projection of Eq. 7).  Normal: with a = V(x+1, y) - V and
 * b = V(x, y+1) - V (all three valid), n = b x a (each component a product
 * minus a product), which with x right, y down, z forward faces the camera,
 * divided by |n| = sqrtf(n . n); pixels on the last row or column, next to an
 * invalid pixel or with |n| = 0 have no normal (all zero).  Maps are
 * row-major, 3 floats per pixel, camera frame. */
void orc_icp_maps(const float* d, int w, int h, const float Kl[9], float* V, float* N) {
    const float ix = (float)(1.0 / (double)Kl[0]), iy = (float)(1.0 / (double)Kl[4]);
    const float ox = (float)(-(double)Kl[2] / (double)Kl[0]), oy = (float)(-(double)Kl[5] / (double)Kl[4]);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const float z = d[(size_t)y * w + x];
            float* v = V + 3 * ((size_t)y * w + x);
            v[0] = z * fmaf(ix, (float)x, ox);
            v[1] = z * fmaf(iy, (float)y, oy);
            v[2] = z;
        }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            float* n = N + 3 * ((size_t)y * w + x);
            n[0] = n[1] = n[2] = 0.0f;
            if (x + 1 >= w || y + 1 >= h) continue;
            const float* v0 = V + 3 * ((size_t)y * w + x);
            const float* v1 = V + 3 * ((size_t)y * w + x + 1);
            const float* v2 = V + 3 * ((size_t)(y + 1) * w + x);
            if (v0[2] == 0.0f || v1[2] == 0.0f || v2[2] == 0.0f) continue;
            const float a[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
            const float b[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
            const float c[3] = {b[1] * a[2] - b[2] * a[1], b[2] * a[0] - b[0] * a[2], b[0] * a[1] - b[1] * a[0]};
            const float len = sqrtf(fmaf(c[0], c[0], fmaf(c[1], c[1], c[2] * c[2])));
            if (!(len > 0.0f)) continue;
            for (int k = 0; k < 3; ++k) n[k] = c[k] / len;
        }
}

/* ------------------------------------------------------ one linear system -- */
typedef struct {
    int32_t w, h;            /* level size */
    float Kl[9];             /* level intrinsics (pinhole) */
    const float* V;          /* current vertex map, camera frame (orc_icp_maps) */
    const float* N;          /* current normal map */
    const float* PV;         /* predicted vertex map, world frame, ray-cast from the previous pose */
    const float* PN;         /* predicted normal map, world frame (zero: no prediction) */
    float R[9], t[3];        /* current pose estimate, camera -> world (binary32) */
    float Rp[9], tp[3];      /* world -> camera of the prediction (binary32) */
    float max_dist2;         /* squared distance gate (m^2) */
    float min_cos;           /* normal-angle gate: cosine of the largest angle */
} orc_icp_level;

static void rigid3(const float R[9], const float t[3], const float p[3], float o[3]) {
    for (int r = 0; r < 3; ++r) o[r] = fmaf(R[r * 3], p[0], fmaf(R[r * 3 + 1], p[1], fmaf(R[r * 3 + 2], p[2], t[r])));
}

/* Projective association and the point-to-plane terms of one level.  For
 * every current pixel u with a vertex and a normal:
 *   p = R V(u) + t (world), m = R N(u);
 *   the prediction pixel: q_c = Rp p + tp, projected with Kl (x = fmaf(fx, X,
 *   cx Z) * (1/Z), likewise y; Z > 0), nearest pixel floor(x + 1/2), inside
 *   the level image, with a prediction there (predicted normal non-zero);
 *   q = PV, nq = PN at that pixel;
 *   gates: |p - q|^2 <= max_dist2 (fmaf chain) and m . nq >= min_cos;
 *   r = (p - q) . nq, J = (nq, p x nq) for xi = (rho, phi) in
 *   T <- exp(xi^) T (d/drho (p + rho) . nq = nq, d/dphi (phi x p) . nq = p x nq).
 * Accumulates, in binary64 and pixel order, A = sum J J^T (36 entries,
 * row-major), g = sum J r, the sum of r^2 and the count.  Returns the count. */
long long orc_icp_system(const orc_icp_level* L, double A[36], double g[6], double* err2) {
    memset(A, 0, 36 * sizeof(double));
    memset(g, 0, 6 * sizeof(double));
    *err2 = 0.0;
    long long n = 0;
    const int w = L->w, h = L->h;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            const float* v = L->V + 3 * i;
            const float* nv = L->N + 3 * i;
            if (v[2] == 0.0f || (nv[0] == 0.0f && nv[1] == 0.0f && nv[2] == 0.0f)) continue;
            float p[3], m[3], qc[3];
            rigid3(L->R, L->t, v, p);
            const float zero[3] = {0.0f, 0.0f, 0.0f};
            rigid3(L->R, zero, nv, m);
            rigid3(L->Rp, L->tp, p, qc);
            if (!(qc[2] > 0.0f)) continue;
            const float rz = 1.0f / qc[2];
            const float ux = fmaf(L->Kl[0], qc[0], L->Kl[2] * qc[2]) * rz;
            const float uy = fmaf(L->Kl[4], qc[1], L->Kl[5] * qc[2]) * rz;
            const float fu = floorf(ux + 0.5f), fv = floorf(uy + 0.5f);
            if (!(fu >= 0.0f && fu <= (float)(w - 1) && fv >= 0.0f && fv <= (float)(h - 1))) continue;
            const size_t j = (size_t)fv * w + (size_t)fu;
            const float* q = L->PV + 3 * j;
            const float* nq = L->PN + 3 * j;
            if (nq[0] == 0.0f && nq[1] == 0.0f && nq[2] == 0.0f) continue;
            const float e[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
            if (fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2])) > L->max_dist2) continue;
            if (!(fmaf(m[0], nq[0], fmaf(m[1], nq[1], m[2] * nq[2])) >= L->min_cos)) continue;
            const float r = fmaf(e[0], nq[0], fmaf(e[1], nq[1], e[2] * nq[2]));
            const float J[6] = {nq[0], nq[1], nq[2], p[1] * nq[2] - p[2] * nq[1], p[2] * nq[0] - p[0] * nq[2],
                                p[0] * nq[1] - p[1] * nq[0]};
            for (int a = 0; a < 6; ++a) {
                for (int b = 0; b < 6; ++b) A[a * 6 + b] += (double)J[a] * (double)J[b];
                g[a] += (double)J[a] * (double)r;
            }
            *err2 += (double)r * (double)r;
            ++n;
        }
    return n;
}

/* ------------------------------------------------------------- solve ---- */
/* xi = -A^-1 g by Cholesky (A = L L^T), binary64.  Returns 0 (xi untouched)
 * when A is not positive definite. */
int orc_icp_solve(const double A[36], const double g[6], double xi[6]) {
    double L[36] = {0};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * 6 + j];
            for (int k = 0; k < j; ++k) s -= L[i * 6 + k] * L[j * 6 + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[i * 6 + i] = sqrt(s);
            } else {
                L[i * 6 + j] = s / L[j * 6 + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[i * 6 + k] * y[k];
        y[i] = s / L[i * 6 + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k * 6 + i] * xi[k];
        xi[i] = s / L[i * 6 + i];
    }
    return 1;
}

/* T <- exp(xi^) T (row-major 4x4, binary64), xi = (rho, phi): Rodrigues for
 * the rotation, V(phi) rho for the translation. */
void orc_icp_update(const double xi[6], double T[16]) {
    const double* rho = xi;
    const double* phi = xi + 3;
    const double a2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], a = sqrt(a2);
    double A, B, C;
    if (a < 1e-4) {
        A = 1.0 - a2 / 6.0;
        B = 0.5 - a2 / 24.0;
        C = 1.0 / 6.0 - a2 / 120.0;
    } else {
        A = sin(a) / a;
        B = (1.0 - cos(a)) / a2;
        C = (a - sin(a)) / (a2 * a);
    }
    const double W[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double W2[9], R[9], Vm[9], t[3], out[16];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += W[i * 3 + k] * W[k * 3 + j];
            W2[i * 3 + j] = s;
        }
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * W[i] + B * W2[i];
        Vm[i] = I + B * W[i] + C * W2[i];
    }
    for (int i = 0; i < 3; ++i) t[i] = Vm[i * 3] * rho[0] + Vm[i * 3 + 1] * rho[1] + Vm[i * 3 + 2] * rho[2];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[i * 3 + k] * T[k * 4 + j];
            out[i * 4 + j] = s + (j == 3 ? t[i] : 0.0);
        }
    }
    for (int j = 0; j < 12; ++j) T[j] = out[j];
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}
