// Layout conversion between the brick-major device volumes and linear
// x-fastest arrays (read-out / restore), and brick summaries of a restored
// volume.
#include <cfloat>
#include <cstdint>

#include "common.cuh"

namespace tsdf {
namespace {

template <typename T, bool TO_LINEAR>
__global__ void __launch_bounds__(256) k_convert(T* brick, T* lin, int nx, int ny, int z0, int64_t n, int nbx,
                                                 int nby) {
    const int32_t nb[3] = {nbx, nby, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = z0 + (int)(i / ((int64_t)nx * ny));
        const int64_t o = brick_offset(x, y, z, nb);
        if (TO_LINEAR)
            lin[i] = brick[o];
        else
            brick[o] = lin[i];
    }
}

template <typename T, bool TO_LINEAR>
cudaError_t convert(T* brick, T* lin, const int32_t dims[3], int z0, int z1, cudaStream_t stream) {
    const int64_t n = (int64_t)dims[0] * dims[1] * (z1 - z0);
    if (n <= 0) return cudaSuccess;
    const int nbx = (dims[0] + BRICK - 1) / BRICK, nby = (dims[1] + BRICK - 1) / BRICK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_convert<T, TO_LINEAR><<<(unsigned)blocks, 256, 0, stream>>>(brick, lin, dims[0], dims[1], z0, n, nbx, nby);
    return cudaGetLastError();
}

// One block per brick: min/max of F over observed voxels and min of w over
// in-volume voxels (the same summary the geometry kernel maintains).
__global__ void __launch_bounds__(128) k_summaries(const float* __restrict__ F, const uint8_t* __restrict__ W,
                                                   BrickSummary* __restrict__ summ, int nx, int ny, int nz, int nbx,
                                                   int nby, float band) {
    __shared__ float s_fmin[4], s_fmax[4];
    __shared__ uint32_t s_wmin[4], s_flags[4];
    const uint32_t b = blockIdx.x;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int tid = threadIdx.x;
    const int lx = (tid & 1) * 4, ly = (tid >> 1) & 7, lz = tid >> 4;
    const size_t base = (size_t)b * BRICK_VOX + (size_t)tid * 4;
    float fmn = FLT_MAX, fmx = -FLT_MAX;
    uint32_t wmn = 0xFFFFFFFFu, flags = 0;
    const float lo_thr = band + CELL_EPS, hi_thr = -band - CELL_EPS;
    for (int j = 0; j < 4; ++j) {
        const int x = bx * BRICK + lx + j, y = by * BRICK + ly, z = bz * BRICK + lz;
        if (x >= nx || y >= ny || z >= nz) continue;
        const uint32_t w = W[base + j];
        const float f = F[base + j];
        wmn = min(wmn, w);
        if (w) { fmn = fminf(fmn, f); fmx = fmaxf(fmx, f); }
        flags |= band_flags(w != 0u, f, lo_thr, hi_thr, lx + j, ly, lz);
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    for (int o = 16; o > 0; o >>= 1) {
        fmn = fminf(fmn, __shfl_xor_sync(0xffffffffu, fmn, o));
        fmx = fmaxf(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
    }
    wmn = __reduce_min_sync(0xffffffffu, wmn);
    if ((tid & 31) == 0) {
        s_fmin[tid >> 5] = fmn;
        s_fmax[tid >> 5] = fmx;
        s_wmin[tid >> 5] = wmn;
        s_flags[tid >> 5] = flags;
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < 4; ++i) {
            fmn = fminf(fmn, s_fmin[i]);
            fmx = fmaxf(fmx, s_fmax[i]);
            wmn = min(wmn, s_wmin[i]);
            flags |= s_flags[i];
        }
        BrickSummary s;
        s.fmin = fmn == FLT_MAX ? __int_as_float(0x7f800000) : fmn;
        s.fmax = fmx == -FLT_MAX ? __int_as_float(0xff800000) : fmx;
        s.wmin = wmn == 0xFFFFFFFFu ? 0u : wmn;
        s.flags = flags;
        summ[b] = s;
    }
}

}  // namespace

cudaError_t launch_to_linear_f32(const float* b, float* l, const int32_t d[3], int z0, int z1, cudaStream_t s) {
    return convert<float, true>(const_cast<float*>(b), l, d, z0, z1, s);
}
cudaError_t launch_to_linear_u8(const uint8_t* b, uint8_t* l, const int32_t d[3], int z0, int z1, cudaStream_t s) {
    return convert<uint8_t, true>(const_cast<uint8_t*>(b), l, d, z0, z1, s);
}
cudaError_t launch_to_linear_u32(const uint32_t* b, uint32_t* l, const int32_t d[3], int z0, int z1, cudaStream_t s) {
    return convert<uint32_t, true>(const_cast<uint32_t*>(b), l, d, z0, z1, s);
}
cudaError_t launch_from_linear_f32(float* b, const float* l, const int32_t d[3], int z0, int z1, cudaStream_t s) {
    return convert<float, false>(b, const_cast<float*>(l), d, z0, z1, s);
}
cudaError_t launch_from_linear_u8(uint8_t* b, const uint8_t* l, const int32_t d[3], int z0, int z1, cudaStream_t s) {
    return convert<uint8_t, false>(b, const_cast<uint8_t*>(l), d, z0, z1, s);
}
cudaError_t launch_from_linear_u32(uint32_t* b, const uint32_t* l, const int32_t d[3], int z0, int z1,
                                   cudaStream_t s) {
    return convert<uint32_t, false>(b, const_cast<uint32_t*>(l), d, z0, z1, s);
}

cudaError_t launch_recompute_summaries(const float* F, const uint8_t* W, BrickSummary* summ, const int32_t ng[3],
                                       float band, cudaStream_t stream) {
    const int nbx = (ng[0] + BRICK - 1) / BRICK, nby = (ng[1] + BRICK - 1) / BRICK, nbz = (ng[2] + BRICK - 1) / BRICK;
    const int64_t nbt = (int64_t)nbx * nby * nbz;
    if (nbt > 0) k_summaries<<<(unsigned)nbt, 128, 0, stream>>>(F, W, summ, ng[0], ng[1], ng[2], nbx, nby, band);
    return cudaGetLastError();
}

}  // namespace tsdf
