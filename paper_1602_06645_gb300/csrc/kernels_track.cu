// Camera tracking (Section III: the KinectFusion loop the paper builds on):
// a depth pyramid with its vertex and normal maps, projective data
// association against the surface predicted by ray casting the geometry
// volume, and point-to-plane Gauss-Newton steps T <- exp(xi^) T.  Operation
// order as stated in tsdf.h (tsdf_track); compiled with --fmad=false so only
// the written fmaf() fuse.  The normal equations are reduced in binary64 in a
// fixed order, and solved and applied on the device, so every step of a
// frame is queued without a host round trip.
#include <cstdint>

#include "common.cuh"

namespace tsdf {
namespace {

constexpr int TRACK_THREADS = 256;

// ------------------------------------------------------------ pyramid ----
__global__ void k_depth_metres(const uint16_t* __restrict__ depth, int n, float* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint32_t D = depth[i];
        d[i] = D ? (float)D * 0.001f : 0.0f;
    }
}

// Level l + 1 pixel from the 2 x 2 block of level l, in the order (0,0),
// (1,0), (0,1), (1,1): the mean of the valid depths within 0.03 m of the
// block's first valid depth, summed in that order.
__global__ void k_pyr_down(const float* __restrict__ src, int w, float* __restrict__ dst, int w2, int h2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w2 || y >= h2) return;
    float first = 0.0f, sum = 0.0f;
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = src[(size_t)(2 * y + (k >> 1)) * w + 2 * x + (k & 1)];
        if (d == 0.0f) continue;
        if (n == 0) first = d;
        if (fabsf(d - first) <= 0.03f) {
            sum = sum + d;
            ++n;
        }
    }
    dst[(size_t)y * w2 + x] = n ? __fdiv_rn(sum, (float)n) : 0.0f;
}

// Vertex d (fmaf(1/fx, x, -cx/fx), fmaf(1/fy, y, -cy/fy), 1) of pixel (x, y).
__device__ __forceinline__ float3 vertex_at(const float* __restrict__ d, int w, int x, int y, const float4 ki) {
    const float z = d[(size_t)y * w + x];
    return make_float3(z * fmaf(ki.x, (float)x, ki.z), z * fmaf(ki.y, (float)y, ki.w), z);
}

// Vertex and normal maps (camera frame): n = b x a with a = V(x+1, y) - V,
// b = V(x, y+1) - V, divided by sqrt(n . n); no normal on the last row or
// column, next to a pixel without depth, or when |n| = 0.
__global__ void k_maps(const float* __restrict__ d, int w, int h, float4 ki, float* __restrict__ V,
                       float* __restrict__ N) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w || y >= h) return;
    const size_t i = (size_t)y * w + x;
    const float3 v0 = vertex_at(d, w, x, y, ki);
    V[3 * i] = v0.x;
    V[3 * i + 1] = v0.y;
    V[3 * i + 2] = v0.z;
    float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
    if (x + 1 < w && y + 1 < h && v0.z != 0.0f) {
        const float3 v1 = vertex_at(d, w, x + 1, y, ki), v2 = vertex_at(d, w, x, y + 1, ki);
        if (v1.z != 0.0f && v2.z != 0.0f) {
            const float a0 = v1.x - v0.x, a1 = v1.y - v0.y, a2 = v1.z - v0.z;
            const float b0 = v2.x - v0.x, b1 = v2.y - v0.y, b2 = v2.z - v0.z;
            const float c0 = b1 * a2 - b2 * a1, c1 = b2 * a0 - b0 * a2, c2 = b0 * a1 - b1 * a0;
            const float len = __fsqrt_rn(fmaf(c0, c0, fmaf(c1, c1, c2 * c2)));
            if (len > 0.0f) {
                n0 = __fdiv_rn(c0, len);
                n1 = __fdiv_rn(c1, len);
                n2 = __fdiv_rn(c2, len);
            }
        }
    }
    N[3 * i] = n0;
    N[3 * i + 1] = n1;
    N[3 * i + 2] = n2;
}

// ------------------------------------------------------ normal equations --
// Sums of one step: the 21 entries of the upper triangle of A = sum J J^T
// (row by row), g = sum J r (6), sum r^2 and the count.
constexpr int NSUM = 29;

__device__ __forceinline__ void rigid3(const float* R, const float* t, float x, float y, float z, float& X, float& Y,
                                       float& Z) {
    X = fmaf(R[0], x, fmaf(R[1], y, fmaf(R[2], z, t[0])));
    Y = fmaf(R[3], x, fmaf(R[4], y, fmaf(R[5], z, t[1])));
    Z = fmaf(R[6], x, fmaf(R[7], y, fmaf(R[8], z, t[2])));
}

// Per pixel: p = R V + t, m = R N; the prediction pixel of Rp p + tp through
// Kl (nearest, inside, Z > 0, with a predicted normal); the distance and
// normal gates; r = (p - q) . nq and J = (nq, p x nq).  The pose of the step
// is read from the device (binary64, rounded once to binary32 here).  Each
// block writes its binary64 partial sums, threads combined in a fixed order.
__global__ void __launch_bounds__(TRACK_THREADS) k_icp_terms(TrackLevel L, const double* __restrict__ pose,
                                                             double* __restrict__ partials) {
    float R[9], t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int k = 0; k < 3; ++k) R[r * 3 + k] = (float)pose[r * 4 + k];
        t[r] = (float)pose[r * 4 + 3];
    }
    double acc[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; ++k) acc[k] = 0.0;
    const int npx = L.w * L.h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += gridDim.x * blockDim.x) {
        const float vx = L.V[3 * i], vy = L.V[3 * i + 1], vz = L.V[3 * i + 2];
        const float nx = L.N[3 * i], ny = L.N[3 * i + 1], nz = L.N[3 * i + 2];
        if (vz == 0.0f || (nx == 0.0f && ny == 0.0f && nz == 0.0f)) continue;
        float p[3], m[3], qc[3];
        rigid3(R, t, vx, vy, vz, p[0], p[1], p[2]);
        const float zero[3] = {0.0f, 0.0f, 0.0f};
        rigid3(R, zero, nx, ny, nz, m[0], m[1], m[2]);
        rigid3(L.Rp, L.tp, p[0], p[1], p[2], qc[0], qc[1], qc[2]);
        if (!(qc[2] > 0.0f)) continue;
        const float rz = __frcp_rn(qc[2]);
        const float ux = fmaf(L.K[0], qc[0], L.K[2] * qc[2]) * rz;
        const float uy = fmaf(L.K[4], qc[1], L.K[5] * qc[2]) * rz;
        const float fu = floorf(ux + 0.5f), fv = floorf(uy + 0.5f);
        if (!(fu >= 0.0f && fu <= (float)(L.w - 1) && fv >= 0.0f && fv <= (float)(L.h - 1))) continue;
        const size_t j = (size_t)fv * L.w + (size_t)fu;
        const float q0 = L.PV[3 * j], q1 = L.PV[3 * j + 1], q2 = L.PV[3 * j + 2];
        const float n0 = L.PN[3 * j], n1 = L.PN[3 * j + 1], n2 = L.PN[3 * j + 2];
        if (n0 == 0.0f && n1 == 0.0f && n2 == 0.0f) continue;
        const float e0 = p[0] - q0, e1 = p[1] - q1, e2 = p[2] - q2;
        if (fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) > L.max_dist2) continue;
        if (!(fmaf(m[0], n0, fmaf(m[1], n1, m[2] * n2)) >= L.min_cos)) continue;
        const float r = fmaf(e0, n0, fmaf(e1, n1, e2 * n2));
        const double J[6] = {n0, n1, n2, (double)(p[1] * n2 - p[2] * n1), (double)(p[2] * n0 - p[0] * n2),
                             (double)(p[0] * n1 - p[1] * n0)};
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) acc[k++] += J[a] * J[b];
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[21 + a] += J[a] * (double)r;
        acc[27] += (double)r * (double)r;
        acc[28] += 1.0;
    }
    // block: warp shuffles (fixed pattern), then warps in order
    __shared__ double red[TRACK_THREADS / 32][NSUM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NSUM; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        double v = 0.0;
        for (int w = 0; w < TRACK_THREADS / 32; ++w) v += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * NSUM + threadIdx.x] = v;
    }
}

// ------------------------------------------------------ solve and update --
// One block of eight warps: the blocks' partials summed per sum in a fixed order,
// then thread 0 solves A xi = -g by Cholesky (binary64) and applies
// T <- exp(xi^) T; a matrix that is not positive definite leaves T as it is.
// The step's sums, its starting pose and its xi are recorded at record.
constexpr int SOLVE_THREADS = 256;
__global__ void __launch_bounds__(SOLVE_THREADS) k_icp_solve(const double* __restrict__ partials, int blocks,
                                                              double* __restrict__ pose, double* __restrict__ record) {
    __shared__ double s[NSUM];
    // warp w sums partials w, w + 8, ...: lane l the blocks l, l + 32, ... in
    // order, then the lanes in a fixed shuffle pattern (deterministic)
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < NSUM; k += SOLVE_THREADS / 32) {
        double v = 0.0;
        for (int b = lane; b < blocks; b += 32) v += partials[(size_t)b * NSUM + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s[k] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double A[36], g[6];
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b, ++k) A[a * 6 + b] = A[b * 6 + a] = s[k];
#pragma unroll
    for (int a = 0; a < 6; ++a) g[a] = s[21 + a];
    // record: sums (29), pose before the step (16), xi (6), solved flag (1)
#pragma unroll
    for (int i = 0; i < NSUM; ++i) record[i] = s[i];
#pragma unroll
    for (int i = 0; i < 16; ++i) record[NSUM + i] = pose[i];
    // fully unrolled (the arrays then live in registers, not in local
    // memory); a pivot that is not positive marks the step unsolved and is
    // replaced by 1 so the remaining arithmetic stays finite (its result is
    // not used)
    double Lc[36] = {0.0};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double v = A[i * 6 + j];
#pragma unroll
            for (int q = 0; q < j; ++q) v -= Lc[i * 6 + q] * Lc[j * 6 + q];
            if (i == j) {
                if (!(v > 0.0)) {
                    ok = false;
                    v = 1.0;
                }
                Lc[i * 6 + i] = sqrt(v);
            } else {
                Lc[i * 6 + j] = v / Lc[j * 6 + j];
            }
        }
    double xi[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (ok) {
        double y[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double v = -g[i];
#pragma unroll
            for (int q = 0; q < i; ++q) v -= Lc[i * 6 + q] * y[q];
            y[i] = v / Lc[i * 6 + i];
        }
#pragma unroll
        for (int i = 5; i >= 0; --i) {
            double v = y[i];
#pragma unroll
            for (int q = i + 1; q < 6; ++q) v -= Lc[q * 6 + i] * xi[q];
            xi[i] = v / Lc[i * 6 + i];
        }
        // exp(xi^): Rodrigues rotation, V(phi) rho translation
        const double* rho = xi;
        const double* phi = xi + 3;
        const double a2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], a = sqrt(a2);
        double cA, cB, cC;
        if (a < 1e-4) {
            cA = 1.0 - a2 / 6.0;
            cB = 0.5 - a2 / 24.0;
            cC = 1.0 / 6.0 - a2 / 120.0;
        } else {
            cA = sin(a) / a;
            cB = (1.0 - cos(a)) / a2;
            cC = (a - sin(a)) / (a2 * a);
        }
        const double W[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
        double W2[9], Rm[9], Vm[9], tv[3], out[12];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) v += W[i * 3 + q] * W[q * 3 + j];
                W2[i * 3 + j] = v;
            }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double I = (i % 4 == 0) ? 1.0 : 0.0;
            Rm[i] = I + cA * W[i] + cB * W2[i];
            Vm[i] = I + cB * W[i] + cC * W2[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) tv[i] = Vm[i * 3] * rho[0] + Vm[i * 3 + 1] * rho[1] + Vm[i * 3 + 2] * rho[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) v += Rm[i * 3 + q] * pose[q * 4 + j];
                out[i * 4 + j] = v + (j == 3 ? tv[i] : 0.0);
            }
#pragma unroll
        for (int i = 0; i < 12; ++i) pose[i] = out[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) record[NSUM + 16 + i] = xi[i];
    record[NSUM + 22] = ok ? 1.0 : 0.0;
}

}  // namespace

cudaError_t launch_track_pyramid(const uint16_t* depth, int W, int H, int levels, float* const* d,
                                 cudaStream_t stream) {
    k_depth_metres<<<(W * H + 255) / 256, 256, 0, stream>>>(depth, W * H, d[0]);
    int w = W, h = H;
    for (int l = 1; l < levels; ++l) {
        const int w2 = w / 2, h2 = h / 2;
        const dim3 blk(32, 8), grd((w2 + 31) / 32, (h2 + 7) / 8);
        k_pyr_down<<<grd, blk, 0, stream>>>(d[l - 1], w, d[l], w2, h2);
        w = w2;
        h = h2;
    }
    return cudaGetLastError();
}

cudaError_t launch_track_maps(const float* d, int w, int h, const float Kinv4[4], float* V, float* N,
                              cudaStream_t stream) {
    const dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
    k_maps<<<grd, blk, 0, stream>>>(d, w, h, make_float4(Kinv4[0], Kinv4[1], Kinv4[2], Kinv4[3]), V, N);
    return cudaGetLastError();
}

// Blocks of a terms launch: one thread per pixel up to TRACK_MAX_BLOCKS
// blocks, then each thread takes several pixels.  Each block reduces its 29
// binary64 sums across its threads; with more blocks that reduction, not the
// pixels, became the kernel's main cost (measured per tracked frame: 1024
// blocks 4.34 ms, 608 and 320 4.35-4.38 ms, 152 3.88 ms, 114 3.96 ms, 76
// 4.05 ms).
constexpr int TRACK_MAX_BLOCKS = 152;  // one per SM of a GB300
int track_blocks(int npx) {
    const int want = (npx + TRACK_THREADS - 1) / TRACK_THREADS;
    return want < TRACK_MAX_BLOCKS ? (want > 0 ? want : 1) : TRACK_MAX_BLOCKS;
}

size_t track_record_doubles() { return NSUM + 16 + 6 + 1; }

cudaError_t launch_track_step(const TrackLevel& L, double* pose, double* partials, double* record,
                              cudaStream_t stream) {
    const int blocks = track_blocks(L.w * L.h);
    k_icp_terms<<<blocks, TRACK_THREADS, 0, stream>>>(L, pose, partials);
    k_icp_solve<<<1, SOLVE_THREADS, 0, stream>>>(partials, blocks, pose, record);
    return cudaGetLastError();
}

}  // namespace tsdf
