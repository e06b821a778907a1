// Mesh extraction from the geometry volume (marching cubes, or marching
// tetrahedra as an option) and per-polygon texture maps from the colour
// volume (Section IV.C-D, Eq. 11-14).  Definitions (operation order, cases,
// orientation, map layout) as stated in tsdf.h; compiled with --fmad=false so
// only the written fmaf() fuse.
#include <cfloat>
#include <cstdint>

#include "common.cuh"
#include "device_math.cuh"

namespace tsdf {
namespace {

constexpr int MESH_THREADS = 128;  // 4 warps, one candidate brick per warp
constexpr int TILE_M = BRICK + 1;  // cells of a brick need one more voxel on the + sides
constexpr int TILE_M3 = TILE_M * TILE_M * TILE_M;

// Corner orders of the six tetrahedra of a cell (main-diagonal split): for the
// axis orderings (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x) the path
// 0, 0 + a0, 0 + a0 + a1, 7.
__device__ __forceinline__ void tet_corners(int t, int c[4]) {
    const int a0 = t < 2 ? 0 : (t < 4 ? 1 : 2);
    const int a1 = (t == 0 || t == 5) ? 1 : ((t == 1 || t == 3) ? 2 : 0);
    c[0] = 0;
    c[1] = 1 << a0;
    c[2] = c[1] | (1 << a1);
    c[3] = 7;
}

// Marching-cubes case table (built on the host from the rules in tsdf.h):
// entry m, for the mask m of inside corners, holds the triangle count and
// then three cell-edge numbers per triangle.
__constant__ uint8_t c_cube_cases[256][16];

// Lower and upper corner of cell edge e = 4 a + r: the lower corner is r with
// a zero bit inserted at position a.
__device__ __forceinline__ void cube_edge_corners(int e, int& p, int& q) {
    const int a = e >> 2, r = e & 3;
    p = a == 0 ? r << 1 : (a == 1 ? (r & 1) | ((r & 2) << 1) : r);
    q = p | (1 << a);
}

// ------------------------------------------------------- candidate bricks --
// A brick holds cells (min corner in the brick) whose corners span it and its
// +x/+y/+z neighbours; some cell can have triangles only if among those
// bricks' observed voxels there is one with F < 0 and one with F >= 0.
__global__ void __launch_bounds__(256) k_mesh_bricks(MeshConst c, const BrickSummary* __restrict__ summ,
                                                     uint32_t* __restrict__ list, uint32_t* __restrict__ n_list) {
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    bool cand = false;
    if (b < nbt) {
        const int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        float mn = FLT_MAX, mx = -FLT_MAX;
        bool any = false;
        for (int k = 0; k < 8; ++k) {
            const int x = bx + (k & 1), y = by + ((k >> 1) & 1), z = bz + (k >> 2);
            if (x >= c.nb[0] || y >= c.nb[1] || z >= c.nb[2]) continue;
            const BrickSummary s = summ[((size_t)z * c.nb[1] + y) * c.nb[0] + x];
            if (!(s.fmin <= FLT_MAX)) continue;  // no observed voxel
            any = true;
            mn = fminf(mn, s.fmin);
            mx = fmaxf(mx, s.fmax);
        }
        cand = any && mn < 0.0f && mx >= 0.0f;
    }
    append(cand, b, n_list, list);
}

struct MeshSlot {
    float F[TILE_M3];
    uint8_t W[TILE_M3];
};

__device__ __forceinline__ float centre_of(const MeshConst& c, int a, int i) {
    return fmaf((float)i + 0.5f, c.s_g, c.origin[a]);
}

// Vertex on the edge between cell corners a and b (p the lower corner index,
// which is the lower linear voxel index).
__device__ __forceinline__ void edge_vertex(const MeshConst& c, const int base[3], const float Fc[8], int a, int b,
                                            float out[3]) {
    const int p = min(a, b), q = max(a, b);
    const float t = __fdiv_rn(Fc[p], Fc[p] - Fc[q]);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float Pp = centre_of(c, ax, base[ax] + ((p >> ax) & 1));
        const float Pq = centre_of(c, ax, base[ax] + ((q >> ax) & 1));
        out[ax] = fmaf(t, Pq - Pp, Pp);
    }
}

// Orient (normal toward the outside corner) and store one triangle.
__device__ __forceinline__ void emit(const MeshConst& c, const int base[3], const float v0[3], const float v1[3],
                                     const float v2[3], int cin, int cout, float* __restrict__ dst) {
    float e1[3], e2[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e1[a] = v1[a] - v0[a];
        e2[a] = v2[a] - v0[a];
        d[a] = centre_of(c, a, base[a] + ((cout >> a) & 1)) - centre_of(c, a, base[a] + ((cin >> a) & 1));
    }
    const float n0 = e1[1] * e2[2] - e1[2] * e2[1];
    const float n1 = e1[2] * e2[0] - e1[0] * e2[2];
    const float n2 = e1[0] * e2[1] - e1[1] * e2[0];
    const bool flip = fmaf(n0, d[0], fmaf(n1, d[1], n2 * d[2])) < 0.0f;
    const float* a1 = flip ? v2 : v1;
    const float* a2 = flip ? v1 : v2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dst[a] = v0[a];
        dst[3 + a] = a1[a];
        dst[6 + a] = a2[a];
    }
}

// Number of triangles of a cell from its corner values (observed cells only).
__device__ __forceinline__ int cell_count(const float Fc[8]) {
    int n = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        int cc[4];
        tet_corners(t, cc);
        int ni = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) ni += Fc[cc[k]] < 0.0f ? 1 : 0;
        n += (ni == 0 || ni == 4) ? 0 : (ni == 2 ? 2 : 1);
    }
    return n;
}

// Write the triangles of one cell from slot `slot` on (those at or beyond cap
// are dropped).
__device__ void cell_emit(const MeshConst& c, const int base[3], const float Fc[8], float* __restrict__ out,
                          uint64_t slot, uint64_t cap) {
    for (int t = 0; t < 6; ++t) {
        int cc[4];
        tet_corners(t, cc);
        int ins[4], outs[4], ni = 0, no = 0;
        for (int k = 0; k < 4; ++k) {
            if (Fc[cc[k]] < 0.0f) ins[ni++] = cc[k];
            else outs[no++] = cc[k];
        }
        if (ni == 0 || no == 0) continue;
        if (ni == 1 || no == 1) {
            const int lone = ni == 1 ? ins[0] : outs[0];
            const int* others = ni == 1 ? outs : ins;
            float v[3][3];
            for (int e = 0; e < 3; ++e) edge_vertex(c, base, Fc, lone, others[e], v[e]);
            if (slot < cap) emit(c, base, v[0], v[1], v[2], ins[0], outs[0], out + 9 * slot);
            ++slot;
        } else {
            float q[4][3];
            edge_vertex(c, base, Fc, ins[0], outs[0], q[0]);
            edge_vertex(c, base, Fc, ins[0], outs[1], q[1]);
            edge_vertex(c, base, Fc, ins[1], outs[1], q[2]);
            edge_vertex(c, base, Fc, ins[1], outs[0], q[3]);
            if (slot < cap) emit(c, base, q[0], q[1], q[2], ins[0], outs[0], out + 9 * slot);
            ++slot;
            if (slot < cap) emit(c, base, q[0], q[2], q[3], ins[0], outs[0], out + 9 * slot);
            ++slot;
        }
    }
}

// Marching cubes: the triangles of one cell from the case table.
__device__ __forceinline__ int cube_count(const float Fc[8]) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) m |= Fc[k] < 0.0f ? 1 << k : 0;
    return c_cube_cases[m][0];
}

__device__ void cube_emit(const MeshConst& c, const int base[3], const float Fc[8], float* __restrict__ out,
                          uint64_t slot, uint64_t cap) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) m |= Fc[k] < 0.0f ? 1 << k : 0;
    const int n = c_cube_cases[m][0];
    for (int t = 0; t < n; ++t, ++slot) {
        if (slot >= cap) continue;
        float* dst = out + 9 * slot;
        for (int k = 0; k < 3; ++k) {
            int p, q;
            cube_edge_corners(c_cube_cases[m][1 + 3 * t + k], p, q);
            edge_vertex(c, base, Fc, p, q, dst + 3 * k);
        }
    }
}

template <bool CUBES>
__global__ void __launch_bounds__(MESH_THREADS) k_mesh(MeshConst c, const float* __restrict__ F,
                                                      const uint8_t* __restrict__ W,
                                                      const uint32_t* __restrict__ list,
                                                      const uint32_t* __restrict__ n_list, float* __restrict__ out,
                                                      uint64_t cap, unsigned long long* __restrict__ count) {
    __shared__ MeshSlot slots[MESH_THREADS / 32];
    MeshSlot& S = slots[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = *n_list;
    for (uint32_t item = warp; item < n; item += nwarps) {
        const uint32_t b = list[item];
        const int bb[3] = {(int)(b % c.nb[0]), (int)((b / c.nb[0]) % c.nb[1]), (int)(b / (c.nb[0] * c.nb[1]))};
        // stage the 9^3 tile: the brick and one voxel more on each + side
        for (int i = lane; i < TILE_M3; i += 32) {
            const int tx = i % TILE_M, ty = (i / TILE_M) % TILE_M, tz = i / (TILE_M * TILE_M);
            const int x = bb[0] * BRICK + tx, y = bb[1] * BRICK + ty, z = bb[2] * BRICK + tz;
            float f = 0.0f;
            uint8_t w = 0;
            if (x < c.ng[0] && y < c.ng[1] && z < c.ng[2]) {
                const int64_t o = brick_offset(x, y, z, c.nb);
                w = W[o];
                f = F[o];
            }
            S.F[i] = f;
            S.W[i] = w;
        }
        __syncwarp();
        // 512 cells, 16 per lane: count, claim slots for the warp, write
        for (int r = 0; r < BRICK_VOX / 32; ++r) {
            const int cell = lane + 32 * r;
            const int cx = cell & 7, cy = (cell >> 3) & 7, cz = cell >> 6;
            const int base[3] = {bb[0] * BRICK + cx, bb[1] * BRICK + cy, bb[2] * BRICK + cz};
            float Fc[8];
            bool obs = base[0] + 1 < c.ng[0] && base[1] + 1 < c.ng[1] && base[2] + 1 < c.ng[2];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = ((cz + (k >> 2)) * TILE_M + cy + ((k >> 1) & 1)) * TILE_M + cx + (k & 1);
                Fc[k] = S.F[i];
                obs = obs && S.W[i] != 0;
            }
            const uint32_t m = obs ? (uint32_t)(CUBES ? cube_count(Fc) : cell_count(Fc)) : 0u;
            uint32_t incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0u) continue;
            unsigned long long wbase = 0;
            if (lane == 0) wbase = atomicAdd(count, (unsigned long long)total);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (m) {
                if (CUBES) cube_emit(c, base, Fc, out, wbase + incl - m, cap);
                else cell_emit(c, base, Fc, out, wbase + incl - m, cap);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ textures ----
constexpr int SCAN_THREADS = 1024;

__device__ __forceinline__ float length3(float x, float y, float z) {
    return __fsqrt_rn(fmaf(x, x, fmaf(y, y, z * z)));
}

__device__ __forceinline__ int map_side(float dist, float size_pixel, int max_side) {
    const float q = floorf(__fdiv_rn(dist, size_pixel) + 0.5f);
    if (!(q >= 2.0f)) return 2;
    if (q > (float)max_side) return max_side;
    return (int)q;
}

// Block-wide exclusive scan of one int64 per thread (the block total is the
// last thread's excl + v).
__device__ void block_scan(int64_t v, int64_t& excl) {
    __shared__ int64_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
        int64_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = si - s;  // exclusive warp offsets
    }
    __syncthreads();
    excl = warp_sums[wid] + incl - v;
    __syncthreads();
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tex_sizes(const float* __restrict__ tris, int64_t n, float size_pixel,
                                                           int32_t max_side, int32_t* __restrict__ wh,
                                                           int64_t* __restrict__ off, int64_t* __restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_THREADS + threadIdx.x;
    int64_t texels = 0;
    if (i < n) {
        const float* T = tris + 9 * i;
        const int w = map_side(length3(T[3] - T[0], T[4] - T[1], T[5] - T[2]), size_pixel, max_side);
        const int h = map_side(length3(T[6] - T[0], T[7] - T[1], T[8] - T[2]), size_pixel, max_side);
        wh[2 * i] = w;
        wh[2 * i + 1] = h;
        texels = (int64_t)w * h;
    }
    int64_t excl;
    block_scan(texels, excl);
    if (i < n) off[i] = excl;
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = excl + texels;
}

// Exclusive scan of the block sums in one block; sums[nb] = grand total.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(int64_t* __restrict__ sums, int64_t nb) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        int64_t excl;
        block_scan(v, excl);
        __shared__ int64_t chunk;
        if (threadIdx.x == SCAN_THREADS - 1) chunk = excl + v;
        __syncthreads();
        if (i < nb) sums[i] = carry + excl;
        carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_tex_offsets(int64_t* __restrict__ off, int64_t n, const int64_t* __restrict__ sums, int64_t nb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += sums[i / SCAN_THREADS];
    if (i == n) off[n] = sums[nb];
}

__device__ __forceinline__ uint32_t texel_colour(const ColourConst& c, const uint32_t* __restrict__ C, float px,
                                                 float py, float pz) {
    const float p[3] = {px, py, pz};
    float f[3];
    int i0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g = fmaf(p[a] - c.origin[a], c.inv_sc, -0.5f);
        const float fl = floorf(g);
        if (!(fl >= -1.0f) || !(fl <= (float)c.nc[a])) return 0u;
        i0[a] = (int)fl;
        f[a] = g - fl;
    }
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, wsum = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = i0[0] + (k & 1), y = i0[1] + ((k >> 1) & 1), z = i0[2] + (k >> 2);
        if (x < 0 || y < 0 || z < 0 || x >= c.nc[0] || y >= c.nc[1] || z >= c.nc[2]) continue;
        const uint32_t col = __ldg(C + brick_offset(x, y, z, c.ncb));
        if ((col >> 24) == 0u) continue;
        float wgt = ((k & 1) ? f[0] : 1.0f - f[0]) * (((k >> 1) & 1) ? f[1] : 1.0f - f[1]);
        wgt = wgt * ((k >> 2) ? f[2] : 1.0f - f[2]);
        acc0 = fmaf(wgt, (float)(col & 0xFFu), acc0);
        acc1 = fmaf(wgt, (float)((col >> 8) & 0xFFu), acc1);
        acc2 = fmaf(wgt, (float)((col >> 16) & 0xFFu), acc2);
        wsum = wsum + wgt;
    }
    if (!(wsum > 0.0f)) return 0u;
    const float acc[3] = {acc0, acc1, acc2};
    uint32_t out = 255u << 24;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float val = floorf(__fdiv_rn(acc[ch], wsum) + 0.5f);
        const uint32_t u = val <= 0.0f ? 0u : (val >= 255.0f ? 255u : (uint32_t)val);
        out |= u << (8 * ch);
    }
    return out;
}

// One thread per texel; its triangle by binary search over the offsets.
__global__ void __launch_bounds__(256) k_tex_fill(ColourConst c, const uint32_t* __restrict__ C,
                                                  const float* __restrict__ tris, int64_t n,
                                                  const int32_t* __restrict__ wh, const int64_t* __restrict__ off,
                                                  int64_t total, uint32_t* __restrict__ texels) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n - 1;  // last t with off[t] <= idx
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= idx) lo = mid;
            else hi = mid - 1;
        }
        const int64_t t = lo;
        const int w = wh[2 * t], h = wh[2 * t + 1];
        const int64_t local = idx - off[t];
        const int j = (int)(local / w), i = (int)(local % w);
        const float* T = tris + 9 * t;
        float p[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float green = __fdiv_rn(T[3 + a] - T[a], (float)(w - 1));
            const float blue = __fdiv_rn(T[6 + a] - T[a], (float)(h - 1));
            p[a] = fmaf((float)j, blue, fmaf((float)i, green, T[a]));
        }
        texels[idx] = texel_colour(c, C, p[0], p[1], p[2]);
    }
}

}  // namespace

cudaError_t upload_cube_cases(const uint8_t (*table)[16], cudaStream_t stream) {
    return cudaMemcpyToSymbolAsync(c_cube_cases, table, sizeof(c_cube_cases), 0, cudaMemcpyHostToDevice, stream);
}

cudaError_t launch_mesh(const MeshConst& c, const float* F, const uint8_t* W, const BrickSummary* summ,
                        uint32_t* list, uint32_t* n_list, float* out, uint64_t cap, unsigned long long* count,
                        bool cubes, cudaStream_t stream) {
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    k_mesh_bricks<<<(nbt + 255) / 256, 256, 0, stream>>>(c, summ, list, n_list);
    int sms = 0, dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cubes) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mesh<true>, MESH_THREADS, 0);
        k_mesh<true><<<max(1, sms * max(1, per_sm)), MESH_THREADS, 0, stream>>>(c, F, W, list, n_list, out, cap,
                                                                               count);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mesh<false>, MESH_THREADS, 0);
        k_mesh<false><<<max(1, sms * max(1, per_sm)), MESH_THREADS, 0, stream>>>(c, F, W, list, n_list, out, cap,
                                                                                count);
    }
    return cudaGetLastError();
}

cudaError_t launch_texture_layout(const float* tris, int64_t n, float size_pixel, int32_t max_side, int32_t* wh,
                                  int64_t* off, int64_t* scratch, cudaStream_t stream) {
    const int64_t nb = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    if (nb > 0) k_tex_sizes<<<(unsigned)nb, SCAN_THREADS, 0, stream>>>(tris, n, size_pixel, max_side, wh, off, scratch);
    k_scan_sums<<<1, SCAN_THREADS, 0, stream>>>(scratch, nb);
    k_tex_offsets<<<(unsigned)((n + 1 + 255) / 256), 256, 0, stream>>>(off, n, scratch, nb);
    return cudaGetLastError();
}

cudaError_t launch_texture_fill(const ColourConst& c, const uint32_t* C, const float* tris, int64_t n,
                                const int32_t* wh, const int64_t* off, int64_t total, uint32_t* texels,
                                cudaStream_t stream) {
    if (total <= 0 || n <= 0) return cudaSuccess;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (total + 255) / 256;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    k_tex_fill<<<grid, 256, 0, stream>>>(c, C, tris, n, wh, off, total, texels);
    return cudaGetLastError();
}

}  // namespace tsdf
