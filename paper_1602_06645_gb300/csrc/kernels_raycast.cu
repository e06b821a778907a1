// Ray casting of the fused volumes (tsdf_raycast): the paper's real-time
// feedback (ray casting both volumes, abstract) and the predicted surface
// vertex map for tracking (ray tracing the geometry volume, Section III).
//
// One thread per pixel, 16x8 pixel blocks (neighbouring rays walk nearby
// bricks, which keeps their gathers in L1/L2).  Operation order as stated in
// tsdf.h; compiled with --fmad=false so only the written fmaf() fuse.
//
// Two exact shortcuts avoid the eight-corner gathers for most samples: when
// all eight corners lie in one brick, that brick's summary decides the sample
// if the brick has no observed voxel (the trilinear value does not exist) or
// is wholly observed with every F equal to 1 (the value is exactly 1, since
// each lerp then computes fmaf(f, 0, 1)).
#include <cfloat>
#include <cstdint>

#include "common.cuh"

namespace tsdf {
namespace {

constexpr int RC_BX = 16, RC_BY = 8;

__device__ __forceinline__ float rc_lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// Trilinear TSDF at world point (px, py, pz); false when it does not exist.
__device__ __forceinline__ bool rc_tsdf(const RayConst& c, const float* __restrict__ F,
                                        const uint8_t* __restrict__ W, const BrickSummary* __restrict__ summ,
                                        float px, float py, float pz, float& out) {
    const float p[3] = {px, py, pz};
    int i0[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g = fmaf(p[a] - c.origin[a], c.inv_sg, -0.5f);
        const float fl = floorf(g);
        if (!(fl >= 0.0f) || !(fl + 1.0f <= (float)(c.ng[a] - 1))) return false;
        i0[a] = (int)fl;
        fr[a] = g - fl;
    }
    if ((i0[0] & 7) != 7 && (i0[1] & 7) != 7 && (i0[2] & 7) != 7) {
        const int64_t b = ((int64_t)(i0[2] >> 3) * c.nb[1] + (i0[1] >> 3)) * c.nb[0] + (i0[0] >> 3);
        const BrickSummary s = summ[b];
        if (!(s.fmin <= FLT_MAX)) return false;  // no observed voxel in the brick
        if (s.wmin > 0u && s.fmin == 1.0f && s.fmax == 1.0f) {
            out = 1.0f;
            return true;
        }
    }
    int64_t off[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) off[k] = brick_offset(i0[0] + (k & 1), i0[1] + ((k >> 1) & 1), i0[2] + (k >> 2), c.nb);
    uint32_t wmin = 255u;
#pragma unroll
    for (int k = 0; k < 8; ++k) wmin = min(wmin, (uint32_t)__ldg(W + off[k]));
    if (wmin == 0u) return false;
    float q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = __ldg(F + off[k]);
    const float c00 = rc_lerp(q[0], q[1], fr[0]), c10 = rc_lerp(q[2], q[3], fr[0]);
    const float c01 = rc_lerp(q[4], q[5], fr[0]), c11 = rc_lerp(q[6], q[7], fr[0]);
    const float c0 = rc_lerp(c00, c10, fr[1]), c1 = rc_lerp(c01, c11, fr[1]);
    out = rc_lerp(c0, c1, fr[2]);
    return true;
}

__global__ void __launch_bounds__(RC_BX * RC_BY) k_raycast(RayConst c, const float* __restrict__ F,
                                                          const uint8_t* __restrict__ W,
                                                          const uint32_t* __restrict__ C,
                                                          const BrickSummary* __restrict__ summ,
                                                          float* __restrict__ range, float* __restrict__ vertex,
                                                          float* __restrict__ normal, uint32_t* __restrict__ rgbw) {
    const int x = blockIdx.x * RC_BX + threadIdx.x, y = blockIdx.y * RC_BY + threadIdx.y;
    if (x >= c.width || y >= c.height) return;
    const float fx = (float)x, fy = (float)y;
    const float dc0 = fmaf(c.Kinv[0], fx, fmaf(c.Kinv[1], fy, c.Kinv[2]));
    const float dc1 = fmaf(c.Kinv[3], fx, fmaf(c.Kinv[4], fy, c.Kinv[5]));
    const float dc2 = fmaf(c.Kinv[6], fx, fmaf(c.Kinv[7], fy, c.Kinv[8]));
    const float nd = __fdiv_rn(1.0f, __fsqrt_rn(fmaf(dc0, dc0, fmaf(dc1, dc1, dc2 * dc2))));
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = fmaf(c.R[3 * a], dc0, fmaf(c.R[3 * a + 1], dc1, c.R[3 * a + 2] * dc2)) * nd;

    float out_t = 0.0f, v[3] = {0.0f, 0.0f, 0.0f}, n[3] = {0.0f, 0.0f, 0.0f};
    uint32_t col = 0u;
    float t = c.near_, tp = 0.0f, Fp = 0.0f;
    bool has_prev = false;
    for (uint32_t it = 0; it < c.max_iter && t <= c.far_; ++it) {
        float Fs;
        const bool ok = rc_tsdf(c, F, W, summ, fmaf(t, d[0], c.t[0]), fmaf(t, d[1], c.t[1]), fmaf(t, d[2], c.t[2]), Fs);
        if (ok && has_prev && Fp > 0.0f && Fs <= 0.0f) {
            const float ts = fmaf(t - tp, __fdiv_rn(Fp, Fp - Fs), tp);
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = fmaf(ts, d[a], c.t[a]);
            out_t = ts;
            float g[3];
            bool good = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float pp[3] = {v[0], v[1], v[2]}, pm[3] = {v[0], v[1], v[2]};
                pp[a] = v[a] + c.s_g;
                pm[a] = v[a] - c.s_g;
                float fp = 0.0f, fm = 0.0f;
                good = good && rc_tsdf(c, F, W, summ, pp[0], pp[1], pp[2], fp) &&
                       rc_tsdf(c, F, W, summ, pm[0], pm[1], pm[2], fm);
                g[a] = fp - fm;
            }
            if (good) {
                const float l2 = fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2]));
                if (l2 > 0.0f) {
                    const float l = __fsqrt_rn(l2);
#pragma unroll
                    for (int a = 0; a < 3; ++a) n[a] = __fdiv_rn(g[a], l);
                }
            }
            if (C) {
                int k[3];
                bool in = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float q = floorf((v[a] - c.origin[a]) * c.inv_sc);
                    in = in && q >= 0.0f && q < (float)c.nc[a];
                    k[a] = in ? (int)q : 0;
                }
                if (in) col = C[brick_offset(k[0], k[1], k[2], c.ncb)];
            }
            break;
        }
        has_prev = ok;
        if (ok) {
            Fp = Fs;
            tp = t;
        }
        t = t + ((ok && Fs < 1.0f) ? c.step_near : c.step_far);
    }
    const size_t i = (size_t)y * c.width + x;
    if (range) range[i] = out_t;
    if (vertex) {
        vertex[3 * i] = v[0];
        vertex[3 * i + 1] = v[1];
        vertex[3 * i + 2] = v[2];
    }
    if (normal) {
        normal[3 * i] = n[0];
        normal[3 * i + 1] = n[1];
        normal[3 * i + 2] = n[2];
    }
    if (rgbw) rgbw[i] = col;
}

}  // namespace

cudaError_t launch_raycast(const RayConst& c, const float* F, const uint8_t* W, const uint32_t* C,
                           const BrickSummary* summ, float* range, float* vertex, float* normal, uint32_t* rgbw,
                           cudaStream_t stream) {
    dim3 block(RC_BX, RC_BY), grid((c.width + RC_BX - 1) / RC_BX, (c.height + RC_BY - 1) / RC_BY);
    k_raycast<<<grid, block, 0, stream>>>(c, F, W, C, summ, range, vertex, normal, rgbw);
    return cudaGetLastError();
}

}  // namespace tsdf
