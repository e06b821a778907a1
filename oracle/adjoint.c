/*
 * CPU ORACLE of the photometric colour loss and its gradient (calibration
 * refinement of the HD camera).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The CUDA path
 * shares no code with it.
 *
 * Problem.  For frames k = 1..n, S_k is the set of colour voxels that pass the
 * depth-side gates of Section IV.B in frame k (Eq. 5-7 and the trilinear TSDF
 * band; orc_record_gates).  S_k does not depend on the HD camera.  With
 * theta = (fx, fy, cx, cy, rho, phi) the HD intrinsics (Eq. 4) and a left
 * perturbation xi = (rho, phi) of the depth-to-HD extrinsic (Eq. 3),
 *   T(xi) = exp(xi^) T0,   P_hd = T(xi) P_vc,   (u, v) = K_hd P_hd / Z_hd,
 * the sample s_k(v) is the bilinear HD intensity at (u, v) (per channel, not
 * rounded), and the fused colour of voxel v is the mean over the frames whose
 * sample lies inside the image: C_v = (1/n_v) sum_k s_k(v) (Eq. 9 with W = 1,
 * in real arithmetic).  The loss against a target volume T is
 *   L = sum_v sum_ch (C_v - T_v)^2   over voxels with n_v > 0 and a target.
 * The discrete choices (S_k, which samples lie inside the image, and the
 * bilinear cell (x0, y0) of each sample) are taken at a reference theta and
 * held fixed, so L is a smooth function of theta and of the image intensities
 * and finite differences converge to the analytic gradient.
 *
 * Everything here is binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_frames, width, height;   /* HD images: n_frames x height x width x 3 */
    const float* images;               /* intensities (binary32 values) */
    const float* Rn;                   /* n_frames x 9: world -> depth camera rotation (binary32 frame constants) */
    const float* tn;                   /* n_frames x 3 */
    const int64_t* offsets;            /* n_frames + 1 offsets into idx */
    const uint32_t* idx;               /* S_k as linear colour indices */
    int32_t nc[3];                     /* colour dims */
    float s_c;                         /* colour voxel edge */
    float origin[3];
    double T0[16];                     /* row-major linearisation point of T_depth_rgb */
} orc_adj;

/* ------------------------------------------------------------ se(3) ---- */
/* exp of xi^ = (rho, phi): R = exp(phi^) (Rodrigues), t = V(phi) rho with
 * V = I + B phi^ + C phi^2, B = (1 - cos a)/a^2, C = (a - sin a)/a^3. */
static void se3_exp(const double xi[6], double R[9], double t[3]) {
    const double* rho = xi;
    const double* phi = xi + 3;
    double a2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double a = sqrt(a2);
    double A, B, C;
    if (a < 1e-4) {  /* Taylor series: avoids the cancellation of 1 - cos a */
        A = 1.0 - a2 / 6.0 + a2 * a2 / 120.0;
        B = 0.5 - a2 / 24.0 + a2 * a2 / 720.0;
        C = 1.0 / 6.0 - a2 / 120.0 + a2 * a2 / 5040.0;
    } else {
        A = sin(a) / a;
        B = (1.0 - cos(a)) / a2;
        C = (a - sin(a)) / (a2 * a);
    }
    double W[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double W2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += W[i * 3 + k] * W[k * 3 + j];
            W2[i * 3 + j] = s;
        }
    double V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * W[i] + B * W2[i];
        V[i] = I + B * W[i] + C * W2[i];
    }
    for (int i = 0; i < 3; ++i) t[i] = V[i * 3] * rho[0] + V[i * 3 + 1] * rho[1] + V[i * 3 + 2] * rho[2];
}

/* --------------------------------------------------------------- pairs -- */
static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* The union V of all S_k, ascending.  Writes it to V (if not NULL) and
 * returns its size. */
int64_t orc_adj_voxels(const orc_adj* P, uint32_t* V) {
    int64_t n = P->offsets[P->n_frames];
    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    memcpy(tmp, P->idx, sizeof(uint32_t) * (size_t)n);
    qsort(tmp, (size_t)n, sizeof(uint32_t), cmp_u32);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (i == 0 || tmp[i] != tmp[i - 1]) tmp[m++] = tmp[i];
    if (V) memcpy(V, tmp, sizeof(uint32_t) * (size_t)m);
    free(tmp);
    return m;
}

static int64_t find_slot(const uint32_t* V, int64_t n, uint32_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (V[mid] == key) return mid;
        if (V[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Camera-space point of pair (k, voxel) in the HD camera at theta: Q = T0 P_vc,
 * P = exp(xi^) Q.  P_vc uses the binary32 frame constants in binary64. */
static void pair_point(const orc_adj* P, int k, uint32_t vox, const double Rx[9], const double tx[3], double Q[3],
                       double Ph[3]) {
    const int nx = P->nc[0], ny = P->nc[1];
    int x = (int)(vox % (uint32_t)nx), y = (int)((vox / (uint32_t)nx) % (uint32_t)ny), z = (int)(vox / ((uint32_t)nx * ny));
    double pw[3] = {P->origin[0] + ((double)x + 0.5) * P->s_c, P->origin[1] + ((double)y + 0.5) * P->s_c,
                    P->origin[2] + ((double)z + 0.5) * P->s_c};
    const float* R = P->Rn + 9 * k;
    const float* t = P->tn + 3 * k;
    double Pc[3];
    for (int r = 0; r < 3; ++r) Pc[r] = R[r * 3] * pw[0] + R[r * 3 + 1] * pw[1] + R[r * 3 + 2] * pw[2] + t[r];
    for (int r = 0; r < 3; ++r)
        Q[r] = P->T0[r * 4] * Pc[0] + P->T0[r * 4 + 1] * Pc[1] + P->T0[r * 4 + 2] * Pc[2] + P->T0[r * 4 + 3];
    for (int r = 0; r < 3; ++r) Ph[r] = Rx[r * 3] * Q[0] + Rx[r * 3 + 1] * Q[1] + Rx[r * 3 + 2] * Q[2] + tx[r];
}

/* Bilinear cells at theta: per pair, (x0, y0) = floor(u, v) when Z > 0 and the
 * 2x2 footprint lies inside the image, else (INT32_MIN, INT32_MIN). */
void orc_adj_cells(const orc_adj* P, const double theta[10], int32_t* cells) {
    double Rx[9], tx[3];
    se3_exp(theta + 4, Rx, tx);
    for (int k = 0; k < P->n_frames; ++k)
        for (int64_t i = P->offsets[k]; i < P->offsets[k + 1]; ++i) {
            double Q[3], Ph[3];
            pair_point(P, k, P->idx[i], Rx, tx, Q, Ph);
            int32_t x0 = INT32_MIN, y0 = INT32_MIN;
            if (Ph[2] > 0) {
                double u = theta[0] * Ph[0] / Ph[2] + theta[2], v = theta[1] * Ph[1] / Ph[2] + theta[3];
                double fx = floor(u), fy = floor(v);
                if (fx >= 0 && fx <= P->width - 2 && fy >= 0 && fy <= P->height - 2) {
                    x0 = (int32_t)fx;
                    y0 = (int32_t)fy;
                }
            }
            cells[2 * i] = x0;
            cells[2 * i + 1] = y0;
        }
}

/* Fused colours, loss and gradients at theta with the cells held fixed.
 *   V, nV        the voxel union (orc_adj_voxels)
 *   target       nV x 3 target colours (NaN = no target), or NULL
 *   C_out, n_out nV x 3 colours and nV sample counts (nullable)
 *   grad         10 gradient entries dL/dtheta, evaluated at xi = 0 (NULL = none)
 *   query, nq    pixel channels (frame, y, x, ch) whose dL/dI is wanted
 *   qgrad        nq gradients (NULL = none)
 * Returns the loss (0 without a target). */
double orc_adj_eval(const orc_adj* P, const double theta[10], const int32_t* cells, const uint32_t* V, int64_t nV,
                    const double* target, double* C_out, int32_t* n_out, double* grad, const int64_t* query,
                    int64_t nq, double* qgrad) {
    const int W = P->width, H = P->height;
    double Rx[9], tx[3];
    se3_exp(theta + 4, Rx, tx);
    double* sum = (double*)calloc((size_t)nV * 3, sizeof(double));
    int32_t* cnt = (int32_t*)calloc((size_t)nV, sizeof(int32_t));
    int64_t npairs = P->offsets[P->n_frames];
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npairs > 0 ? npairs : 1));
    /* forward: C_v = mean of the bilinear samples */
    for (int k = 0; k < P->n_frames; ++k) {
        const float* img = P->images + (size_t)k * H * W * 3;
        for (int64_t i = P->offsets[k]; i < P->offsets[k + 1]; ++i) {
            slot[i] = find_slot(V, nV, P->idx[i]);
            if (cells[2 * i] == INT32_MIN) continue;
            double Q[3], Ph[3];
            pair_point(P, k, P->idx[i], Rx, tx, Q, Ph);
            double u = theta[0] * Ph[0] / Ph[2] + theta[2], v = theta[1] * Ph[1] / Ph[2] + theta[3];
            int x0 = cells[2 * i], y0 = cells[2 * i + 1];
            double ax = u - x0, ay = v - y0;
            const float* p00 = img + ((size_t)y0 * W + x0) * 3;
            const float* p10 = p00 + 3;
            const float* p01 = p00 + (size_t)W * 3;
            const float* p11 = p01 + 3;
            for (int c = 0; c < 3; ++c)
                sum[slot[i] * 3 + c] += (1 - ax) * (1 - ay) * p00[c] + ax * (1 - ay) * p10[c] + (1 - ax) * ay * p01[c] +
                                        ax * ay * p11[c];
            cnt[slot[i]] += 1;
        }
    }
    double loss = 0.0;
    double* g = (double*)calloc((size_t)nV * 3, sizeof(double)); /* dL/ds per voxel and channel */
    for (int64_t s = 0; s < nV; ++s) {
        for (int c = 0; c < 3; ++c) {
            double C = cnt[s] ? sum[s * 3 + c] / cnt[s] : 0.0;
            if (C_out) C_out[s * 3 + c] = C;
            if (target && cnt[s] && !isnan(target[s * 3 + c])) {
                double d = C - target[s * 3 + c];
                loss += d * d;
                g[s * 3 + c] = 2.0 * d / cnt[s];
            }
        }
        if (n_out) n_out[s] = cnt[s];
    }
    /* backward */
    if (grad) {
        for (int j = 0; j < 10; ++j) grad[j] = 0.0;
        for (int k = 0; k < P->n_frames; ++k) {
            const float* img = P->images + (size_t)k * H * W * 3;
            for (int64_t i = P->offsets[k]; i < P->offsets[k + 1]; ++i) {
                if (cells[2 * i] == INT32_MIN) continue;
                const double* gv = g + slot[i] * 3;
                if (gv[0] == 0 && gv[1] == 0 && gv[2] == 0) continue;
                double Q[3], Ph[3];
                pair_point(P, k, P->idx[i], Rx, tx, Q, Ph);
                double X = Ph[0], Y = Ph[1], Z = Ph[2];
                double u = theta[0] * X / Z + theta[2], v = theta[1] * Y / Z + theta[3];
                int x0 = cells[2 * i], y0 = cells[2 * i + 1];
                double ax = u - x0, ay = v - y0;
                const float* p00 = img + ((size_t)y0 * W + x0) * 3;
                const float* p10 = p00 + 3;
                const float* p01 = p00 + (size_t)W * 3;
                const float* p11 = p01 + 3;
                double dsdu = 0, dsdv = 0;  /* sum over channels of g_c * ds_c/du, ds_c/dv */
                for (int c = 0; c < 3; ++c) {
                    dsdu += gv[c] * ((1 - ay) * (p10[c] - p00[c]) + ay * (p11[c] - p01[c]));
                    dsdv += gv[c] * ((1 - ax) * (p01[c] - p00[c]) + ax * (p11[c] - p10[c]));
                }
                /* intrinsics */
                grad[0] += dsdu * X / Z;
                grad[1] += dsdv * Y / Z;
                grad[2] += dsdu;
                grad[3] += dsdv;
                /* dL/dP_hd */
                double dP[3] = {dsdu * theta[0] / Z, dsdv * theta[1] / Z,
                                -(dsdu * theta[0] * X + dsdv * theta[1] * Y) / (Z * Z)};
                /* left perturbation at xi = 0: dP/drho = I, dP/dphi = -[P]x */
                grad[4] += dP[0];
                grad[5] += dP[1];
                grad[6] += dP[2];
                /* dP/dphi_j = e_j x P  ->  dL/dphi = P x dP */
                grad[7] += Y * dP[2] - Z * dP[1];
                grad[8] += Z * dP[0] - X * dP[2];
                grad[9] += X * dP[1] - Y * dP[0];
            }
        }
    }
    if (qgrad) {
        for (int64_t q = 0; q < nq; ++q) {
            int64_t k = query[4 * q], y = query[4 * q + 1], x = query[4 * q + 2], c = query[4 * q + 3];
            double acc = 0.0;
            for (int64_t i = P->offsets[k]; i < P->offsets[k + 1]; ++i) {
                if (cells[2 * i] == INT32_MIN) continue;
                int x0 = cells[2 * i], y0 = cells[2 * i + 1];
                if (x < x0 || x > x0 + 1 || y < y0 || y > y0 + 1) continue;
                double Q[3], Ph[3];
                pair_point(P, (int)k, P->idx[i], Rx, tx, Q, Ph);
                double u = theta[0] * Ph[0] / Ph[2] + theta[2], v = theta[1] * Ph[1] / Ph[2] + theta[3];
                double ax = u - x0, ay = v - y0;
                double wx = (x == x0) ? 1 - ax : ax, wy = (y == y0) ? 1 - ay : ay;
                acc += g[slot[i] * 3 + c] * wx * wy;
            }
            qgrad[q] = acc;
        }
    }
    free(sum);
    free(cnt);
    free(slot);
    free(g);
    return loss;
}

int orc_adj_size(void) { return (int)sizeof(orc_adj); }
