// Photometric colour loss of the fused colour volume and its adjoint, for
// refining the HD camera's calibration (intrinsics of Eq. 4, extrinsic of
// Eq. 3) from the colour consistency of the fused volume.
//
// For every colour voxel v recorded in the sets S_k (frames whose depth-side
// gates it passes), the forward pass is the mean of its binary32 bilinear HD
// samples over the frames where the 2x2 footprint lies inside the image:
//   C_v = (1/n_v) sum_k s_k(v),   s_k = bilinear(I_k, K_hd T P_vc)
// (Eq. 9 with W = 1, unrounded).  The backward pass takes dL/dC_v and returns
// dL/dI_k (scattered to the 4 footprint pixels with atomics), dL/dK_hd and the
// derivative with respect to a left se(3) perturbation of the extrinsic at the
// linearisation point: dP/drho = I, dP/dphi_j = e_j x P.
//
// One thread per voxel slot; a slot's frames are visited in ascending order,
// so the colours are deterministic.  Camera-parameter gradients are reduced
// per block in binary64 and then over blocks in a fixed order.
#include <cstdint>

#include "common.cuh"
#include "device_math.cuh"
#include "ffloat.cuh"

namespace tsdf {
namespace {

constexpr int ADJ_THREADS = 256;

// ------------------------------------------------------------ finalize ----
// Slots: the first pair of a voxel claims it (-1 -> -2) and takes the next
// slot number; the voxel map then holds the slot.
__global__ void k_slot_claim(AdjBuffers a, uint32_t* err) {
    const uint32_t n = min(a.counters[0], a.pair_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = a.pair_vox[i];
        if (atomicCAS(&a.slot_of[v], -1, -2) == -1) {
            const uint32_t s = atomicAdd(&a.counters[1], 1u);
            if (s < a.slot_cap) {
                a.V[s] = v;
                a.slot_of[v] = (int32_t)s;
            } else {
                atomicOr(err, ERR_SLOT_OVERFLOW);
            }
        }
    }
}

__global__ void k_slot_fill(AdjBuffers a, uint32_t* err) {
    const uint32_t n = min(a.counters[0], a.pair_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t s = a.slot_of[a.pair_vox[i]];
        if (s < 0) continue;
        const uint32_t j = atomicAdd(&a.slot_count[s], 1u);
        if (j < (uint32_t)a.max_frames)
            a.slot_frames[(size_t)s * a.max_frames + j] = a.pair_frame[i];
        else
            atomicOr(err, ERR_SLOT_OVERFLOW);
    }
}

// Insertion sort of each slot's frame ids (a frame appears at most once).
__global__ void k_slot_sort(AdjBuffers a) {
    const uint32_t n = min(a.counters[1], a.slot_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint8_t* f = a.slot_frames + (size_t)s * a.max_frames;
        const int m = min((int)a.slot_count[s], a.max_frames);
        for (int i = 1; i < m; ++i) {
            const uint8_t key = f[i];
            int j = i - 1;
            while (j >= 0 && f[j] > key) {
                f[j + 1] = f[j];
                --j;
            }
            f[j + 1] = key;
        }
    }
}

// ------------------------------------------------------------- sample -----
struct Sample {
    bool valid;
    int x0, y0;
    float ax, ay, X, Y, Z;
};

// HD sample position of voxel (centre p) in frame k at the linearisation
// point: P_vc = R_n p + t_n (Eq. 5), P = R P_vc + t (Eq. 3), (u, v) = K P / Z
// (Eq. 4) with the operations of the colour update's projection
// (xh = fmaf(fx, X, cx Z), u = xh * (1/Z)); the bilinear footprint
// (x0..x0+1, y0..y0+1), x0 = floor(u), must lie in the image.  The cell is an
// integer decision, taken exactly as the fusion's bilinear sampling takes it.
__device__ __forceinline__ Sample hd_sample(const AdjCamera& cam, const AdjFrame& fr, float px, float py, float pz) {
    Sample s;
    float Xc, Yc, Zc;
    rigid(fr.R, fr.t, px, py, pz, Xc, Yc, Zc);
    rigid(cam.R, cam.t, Xc, Yc, Zc, s.X, s.Y, s.Z);
    s.valid = false;
    if (!(s.Z > 0.0f)) return s;
    const float rz = __frcp_rn(s.Z);
    const float u = fmaf(cam.fx, s.X, cam.cx * s.Z) * rz, v = fmaf(cam.fy, s.Y, cam.cy * s.Z) * rz;
    const float fx0 = floorf(u), fy0 = floorf(v);
    if (!(fx0 >= 0.0f && fx0 + 1.0f <= (float)(cam.width - 1) && fy0 >= 0.0f && fy0 + 1.0f <= (float)(cam.height - 1)))
        return s;
    s.valid = true;
    s.x0 = (int)fx0;
    s.y0 = (int)fy0;
    return s;
}

// The bilinear fractions (u - x0, v - y0) of a valid sample, from the sample
// position in float-float arithmetic: the voxel centre origin + (k + 1/2) s_c,
// both rigid motions and the projection carry ~48 bits, so the fractions are
// those of the exact position for the given binary32 constants to within a
// few binary32 roundings (binary32 throughout would be ~1e-4 pixel off at
// HD resolution, a visible colour error across a sharp image edge).
__device__ __forceinline__ void hd_fractions(const AdjCamera& cam, const AdjFrame& fr, const int k[3], Sample& s) {
    ff p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = ff_add(two_prod((float)k[a] + 0.5f, cam.s_c), cam.origin[a]);
    ff c[3], h[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) c[r] = ff_row(fr.R + 3 * r, fr.t[r], p);
#pragma unroll
    for (int r = 0; r < 3; ++r) h[r] = ff_row(cam.R + 3 * r, cam.t[r], c);
    const ff qx = ff_div(h[0], h[2]), qy = ff_div(h[1], h[2]);
    const ff u = ff_add(ff_mul(qx, cam.fx), cam.cx), v = ff_add(ff_mul(qy, cam.fy), cam.cy);
    s.ax = (u.hi - (float)s.x0) + u.lo;  // the difference of the high parts is exact (Sterbenz)
    s.ay = (v.hi - (float)s.y0) + v.lo;
}

__device__ __forceinline__ void voxel_index(const AdjCamera& cam, uint32_t lin, int k[3]) {
    const uint32_t nx = (uint32_t)cam.nc[0], ny = (uint32_t)cam.nc[1];
    k[0] = (int)(lin % nx);
    k[1] = (int)((lin / nx) % ny);
    k[2] = (int)(lin / (nx * ny));
}

__device__ __forceinline__ void voxel_centre(const AdjCamera& cam, const int k[3], float& px, float& py, float& pz) {
    px = fmaf((float)k[0] + 0.5f, cam.s_c, cam.origin[0]);
    py = fmaf((float)k[1] + 0.5f, cam.s_c, cam.origin[1]);
    pz = fmaf((float)k[2] + 0.5f, cam.s_c, cam.origin[2]);
}

// ------------------------------------------------------------ forward -----
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_forward(AdjCamera cam, AdjBuffers a, uint32_t n_slots,
                                                             const float* __restrict__ images, float* __restrict__ C,
                                                             int32_t* __restrict__ n_out) {
    const size_t plane = (size_t)cam.height * cam.width * 3;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_slots; s += gridDim.x * blockDim.x) {
        int kv[3];
        float px, py, pz;
        voxel_index(cam, a.V[s], kv);
        voxel_centre(cam, kv, px, py, pz);
        const uint8_t* fl = a.slot_frames + (size_t)s * a.max_frames;
        const int m = min((int)a.slot_count[s], a.max_frames);
        float sum[3] = {0.0f, 0.0f, 0.0f};
        int n = 0;
        for (int j = 0; j < m; ++j) {
            const int k = fl[j];
            Sample smp = hd_sample(cam, a.frames[k], px, py, pz);
            if (!smp.valid) continue;
            hd_fractions(cam, a.frames[k], kv, smp);
            const float* p00 = images + k * plane + ((size_t)smp.y0 * cam.width + smp.x0) * 3;
            const float* p01 = p00 + (size_t)cam.width * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float top = fmaf(smp.ax, p00[3 + ch] - p00[ch], p00[ch]);
                const float bot = fmaf(smp.ax, p01[3 + ch] - p01[ch], p01[ch]);
                sum[ch] += fmaf(smp.ay, bot - top, top);
            }
            ++n;
        }
        const float inv = n ? 1.0f / (float)n : 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) C[(size_t)s * 3 + ch] = sum[ch] * inv;
        n_out[s] = n;
        a.n_valid[s] = n;
    }
}

// ----------------------------------------------------------- backward -----
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_backward(AdjCamera cam, AdjBuffers a, uint32_t n_slots,
                                                              const float* __restrict__ images,
                                                              const float* __restrict__ grad_C,
                                                              float* __restrict__ grad_images) {
    __shared__ double red[ADJ_THREADS / 32][10];
    const size_t plane = (size_t)cam.height * cam.width * 3;
    double acc[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) acc[j] = 0.0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_slots; s += gridDim.x * blockDim.x) {
        const int n = a.n_valid[s];
        if (n == 0) continue;
        const float inv = 1.0f / (float)n;
        const float g[3] = {grad_C[(size_t)s * 3] * inv, grad_C[(size_t)s * 3 + 1] * inv, grad_C[(size_t)s * 3 + 2] * inv};
        if (g[0] == 0.0f && g[1] == 0.0f && g[2] == 0.0f) continue;
        int kv[3];
        float px, py, pz;
        voxel_index(cam, a.V[s], kv);
        voxel_centre(cam, kv, px, py, pz);
        const uint8_t* fl = a.slot_frames + (size_t)s * a.max_frames;
        const int m = min((int)a.slot_count[s], a.max_frames);
        for (int j = 0; j < m; ++j) {
            const int k = fl[j];
            Sample smp = hd_sample(cam, a.frames[k], px, py, pz);
            if (!smp.valid) continue;
            hd_fractions(cam, a.frames[k], kv, smp);
            const size_t o00 = k * plane + ((size_t)smp.y0 * cam.width + smp.x0) * 3;
            const size_t o01 = o00 + (size_t)cam.width * 3;
            const float* p00 = images + o00;
            const float* p01 = images + o01;
            float dsdu = 0.0f, dsdv = 0.0f;
            const float w00 = (1.0f - smp.ax) * (1.0f - smp.ay), w10 = smp.ax * (1.0f - smp.ay);
            const float w01 = (1.0f - smp.ax) * smp.ay, w11 = smp.ax * smp.ay;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                dsdu += g[ch] * ((1.0f - smp.ay) * (p00[3 + ch] - p00[ch]) + smp.ay * (p01[3 + ch] - p01[ch]));
                dsdv += g[ch] * ((1.0f - smp.ax) * (p01[ch] - p00[ch]) + smp.ax * (p01[3 + ch] - p00[3 + ch]));
                atomicAdd(grad_images + o00 + ch, g[ch] * w00);
                atomicAdd(grad_images + o00 + 3 + ch, g[ch] * w10);
                atomicAdd(grad_images + o01 + ch, g[ch] * w01);
                atomicAdd(grad_images + o01 + 3 + ch, g[ch] * w11);
            }
            const float rz = 1.0f / smp.Z;
            const float X = smp.X, Y = smp.Y, Z = smp.Z;
            acc[0] += (double)(dsdu * X * rz);
            acc[1] += (double)(dsdv * Y * rz);
            acc[2] += (double)dsdu;
            acc[3] += (double)dsdv;
            const float dPx = dsdu * cam.fx * rz, dPy = dsdv * cam.fy * rz;
            const float dPz = -(dsdu * cam.fx * X + dsdv * cam.fy * Y) * rz * rz;
            acc[4] += (double)dPx;
            acc[5] += (double)dPy;
            acc[6] += (double)dPz;
            acc[7] += (double)(Y * dPz - Z * dPy);
            acc[8] += (double)(Z * dPx - X * dPz);
            acc[9] += (double)(X * dPy - Y * dPx);
        }
    }
    // block reduction in binary64, fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int w = 0; w < ADJ_THREADS / 32; ++w) v += red[w][threadIdx.x];
        a.partials[(size_t)blockIdx.x * 10 + threadIdx.x] = v;
    }
}

__global__ void k_adj_reduce(AdjBuffers a, int blocks) {
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int b = 0; b < blocks; ++b) v += a.partials[(size_t)b * 10 + threadIdx.x];
        a.grad[threadIdx.x] = v;
    }
}

}  // namespace

cudaError_t launch_adjoint_finalize(const AdjBuffers& a, uint32_t n_pairs_max, cudaStream_t stream) {
    // a.counters[2] is used as the error word of this phase
    const unsigned blocks = n_pairs_max ? (unsigned)((n_pairs_max + 255) / 256 > 4096 ? 4096 : (n_pairs_max + 255) / 256) : 1u;
    k_slot_claim<<<blocks, 256, 0, stream>>>(a, a.counters + 2);
    k_slot_fill<<<blocks, 256, 0, stream>>>(a, a.counters + 2);
    k_slot_sort<<<blocks, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_forward(const AdjCamera& cam, const AdjBuffers& a, uint32_t n_slots, const float* images,
                                   float* C, int32_t* n_out, cudaStream_t stream) {
    if (n_slots == 0) return cudaSuccess;
    unsigned blocks = (n_slots + ADJ_THREADS - 1) / ADJ_THREADS;
    if (blocks > 8192u) blocks = 8192u;
    k_adj_forward<<<blocks, ADJ_THREADS, 0, stream>>>(cam, a, n_slots, images, C, n_out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_backward(const AdjCamera& cam, const AdjBuffers& a, uint32_t n_slots, const float* images,
                                    const float* grad_C, float* grad_images, int blocks, cudaStream_t stream) {
    k_adj_backward<<<blocks, ADJ_THREADS, 0, stream>>>(cam, a, n_slots, images, grad_C, grad_images);
    k_adj_reduce<<<1, 32, 0, stream>>>(a, blocks);
    return cudaGetLastError();
}

}  // namespace tsdf
