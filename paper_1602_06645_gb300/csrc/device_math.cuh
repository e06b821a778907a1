// Device helpers shared by the CUDA translation units: projection (Eq. 1/4/6),
// nearest pixel, rigid motion (Eq. 3/5), back-projection (Eq. 7), lerp and
// warp-aggregated list appends.  Operation order as documented in common.cuh.
#pragma once

#include "common.cuh"

namespace tsdf {

// Eq. 1 / 4 / 6: (xh, yh, zh) = K (X, Y, Z), u = xh * (1/zh), v = yh * (1/zh).
// With a pinhole K (zero skew and bottom row (0, 0, 1)) the zero terms are
// dropped; that changes at most the sign of a zero xh or yh, which rounds to
// the same pixel.
__device__ __forceinline__ bool project(const float* K, int pinhole, float X, float Y, float Z, float& u, float& v) {
    float xh, yh, zh;
    if (pinhole) {
        xh = fmaf(K[0], X, K[2] * Z);
        yh = fmaf(K[4], Y, K[5] * Z);
        zh = Z;
    } else {
        xh = fmaf(K[0], X, fmaf(K[1], Y, K[2] * Z));
        yh = fmaf(K[3], X, fmaf(K[4], Y, K[5] * Z));
        zh = fmaf(K[6], X, fmaf(K[7], Y, K[8] * Z));
    }
    if (!(zh > 0.0f)) return false;
    float rz = __frcp_rn(zh);
    u = xh * rz;
    v = yh * rz;
    return true;
}

// Nearest pixel, half-up: floor(u + 1/2).  With t = u + 1/2, the bounds
// 0 <= floor(t) <= W - 1 are tested in float as 0 <= t < W (NaN fails), and
// only then is t converted with rounding toward minus infinity.
__device__ __forceinline__ bool nearest_pixel(float u, float v, int W, int H, int& iu, int& iv) {
    const float tu = u + 0.5f, tv = v + 0.5f;
    if (!(tu >= 0.0f && tu < (float)W && tv >= 0.0f && tv < (float)H)) return false;
    iu = __float2int_rd(tu);
    iv = __float2int_rd(tv);
    return true;
}

// project() then nearest_pixel() without branches: true with the pixel's
// linear index when the point is in front of the camera and its nearest pixel
// is inside the image (same operations, same rounding); else false, pix = 0.
__device__ __forceinline__ bool project_pixel(const float* K, int pinhole, float X, float Y, float Z, int W, int H,
                                              int& pix) {
    float xh, yh, zh;
    if (pinhole) {
        xh = fmaf(K[0], X, K[2] * Z);
        yh = fmaf(K[4], Y, K[5] * Z);
        zh = Z;
    } else {
        xh = fmaf(K[0], X, fmaf(K[1], Y, K[2] * Z));
        yh = fmaf(K[3], X, fmaf(K[4], Y, K[5] * Z));
        zh = fmaf(K[6], X, fmaf(K[7], Y, K[8] * Z));
    }
    const float rz = __frcp_rn(zh);
    const float tu = xh * rz + 0.5f, tv = yh * rz + 0.5f;
    const bool ok = zh > 0.0f && tu >= 0.0f && tu < (float)W && tv >= 0.0f && tv < (float)H;
    pix = ok ? __float2int_rd(tv) * W + __float2int_rd(tu) : 0;
    return ok;
}

// y = R x + t, row by row as fmaf(R0, x, fmaf(R1, y, fmaf(R2, z, t))).
__device__ __forceinline__ void rigid(const float* R, const float* t, float x, float y, float z, float& X,
                                      float& Y, float& Z) {
    X = fmaf(R[0], x, fmaf(R[1], y, fmaf(R[2], z, t[0])));
    Y = fmaf(R[3], x, fmaf(R[4], y, fmaf(R[5], z, t[1])));
    Z = fmaf(R[6], x, fmaf(R[7], y, fmaf(R[8], z, t[2])));
}

// Back-projection d * K_c^-1 (iu, iv, 1) of a depth pixel (Eq. 7).
__device__ __forceinline__ void back_project(const FrameConst& c, int iu, int iv, float d, float& X, float& Y,
                                             float& Z) {
    float fu = (float)iu, fv = (float)iv;
    if (c.kdi_pinhole) {
        X = d * fmaf(c.Kdi[0], fu, c.Kdi[2]);
        Y = d * fmaf(c.Kdi[4], fv, c.Kdi[5]);
        Z = d;
    } else {
        X = d * fmaf(c.Kdi[0], fu, fmaf(c.Kdi[1], fv, c.Kdi[2]));
        Y = d * fmaf(c.Kdi[3], fu, fmaf(c.Kdi[4], fv, c.Kdi[5]));
        Z = d * fmaf(c.Kdi[6], fu, fmaf(c.Kdi[7], fv, c.Kdi[8]));
    }
}

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// Correctly rounded a / b for the small integer divisor b = w + 1 (1..256),
// given y = RN(1/b): q = RN(a y) is within about an ulp of a / b, the
// residual r = a - b q is exact in one fused multiply-add, and RN(q + r y) is
// the correctly rounded quotient (Markstein's correction step; checked
// exhaustively against the IEEE division for every divisor and every
// significand of a).  Replaces an IEEE division, which costs a range check and
// several dependent instructions more per voxel.  The geometry kernel takes
// y from rcp2_rn below, which equals RN(1/b) over its whole range.
__device__ __forceinline__ float div_by_weight(float a, float b, float y) {
    const float q = a * y;
    const float r = fmaf(-b, q, a);
    return fmaf(r, y, q);
}

// Correctly rounded reciprocals of a pair, 1/z for z in [2^-126, 2^126): the
// hardware's approximate reciprocal (within an ulp) refined by one Newton
// step with a fused residual, y = y0 + y0 (1 - z y0), whose rounding gives
// RN(1/z) over that whole range (checked exhaustively against __frcp_rn).
__device__ __forceinline__ float2 rcp2_rn(float2 z) {
    float2 y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0.x) : "f"(z.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0.y) : "f"(z.y));
    const float2 e = __ffma2_rn(make_float2(-z.x, -z.y), y0, make_float2(1.0f, 1.0f));
    return __ffma2_rn(e, y0, y0);
}

// Entry of a kernel of the per-frame chain.  Launched with programmatic
// stream serialization, a kernel may start while its predecessor drains:
// griddepcontrol.wait holds it until the predecessor grid has completed and
// its writes are visible (a no-op after a normal launch), and
// griddepcontrol.launch_dependents lets the next kernel of the chain be
// scheduled as soon as this one's blocks retire.
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Warp-aggregated append of `pred` items to list[ctr++].
__device__ __forceinline__ void append(bool pred, uint32_t value, uint32_t* ctr, uint32_t* list) {
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (!mask) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

}  // namespace tsdf
