// Per-frame fusion kernels: depth tiles, brick culling, geometry (TSDF)
// update, colour work list and colour update (Section IV.B).
//
// Order per frame on one stream:
//   k_depth_tiles   min / max valid depth of each 8x8 depth tile; zeroes counters
//   k_bricks        conservative per-brick visibility -> geometry and visible lists
//   k_geometry      persistent: TSDF update of each listed brick, brick summaries
//   k_colour_list   visible bricks whose owned cells (the brick and the first layers
//                   of its + neighbours) can hold |F| <= band
//   k_colour_band   one warp per listed brick: stages its geometry tile, finds
//                   the trilinear cells that can pass the band gate and records
//                   the colour voxels whose trilinear TSDF passes it
//   k_colour_voxels one thread per recorded colour voxel: the rest of the update
// Culling only removes work whose every voxel the per-voxel logic would skip
// or leave unchanged, so results do not depend on it.
#include <cfloat>
#include <cstdint>

#include <type_traits>

#include "common.cuh"
#include "device_math.cuh"

namespace tsdf {
namespace {

constexpr int GEO_THREADS = 128;  // 4 voxels per thread, one brick per block iteration
constexpr int COL_THREADS = 128;  // 4 warps, one colour work item per warp
constexpr int TILE_G = BRICK + 1;          // geometry tile edge: the brick + the next bricks' first voxel layer
constexpr int TILE_G3 = TILE_G * TILE_G * TILE_G;
constexpr int CELLS = BRICK;               // trilinear cells a brick owns: lower corner in the brick
constexpr int CELLS3 = CELLS * CELLS * CELLS;

// ------------------------------------------------------- depth tiles ----
// Per 8x8-pixel tile the min / max valid depth (mm); with depth_m, also the
// depth in metres per pixel as the geometry update reads it: RN(D * 0.001),
// -inf where D = 0.  One warp per strip of four tiles (32 x 8 pixels): lane
// x reads column x of the strip row by row (64 contiguous bytes per row),
// and lanes 8t .. 8t + 7 reduce tile t.  Blocks are two warps: the next
// frame's tiles run beside the current frame's colour kernels, whose blocks
// leave only a few thousand registers of an SM free.
constexpr int TILES_THREADS = 64;
constexpr int STRIP_PX = 32;  // strip width: four tiles

__host__ __device__ inline uint32_t depth_strips(const FrameConst& c) {
    return (uint32_t)((c.dw + STRIP_PX - 1) / STRIP_PX) * (uint32_t)c.tiles_y;
}

// Depth tiles of one 32 x 8-pixel strip (four 8 x 8 tiles) by one warp: lane
// x reads column x of the strip's eight rows (eight independent reads, each
// row's 64 bytes coalesced); min / max over the column, then over each group
// of eight lanes.  depth_m (optional) receives the strip's depths in metres.
__device__ __forceinline__ void depth_strip(const FrameConst& c, const uint16_t* __restrict__ depth,
                                            uint32_t* __restrict__ tiles, float* __restrict__ depth_m,
                                            uint32_t strip, int lane) {
    static_assert(TILE_PX == 8 && STRIP_PX == 4 * TILE_PX, "the lane layout below assumes 8x8 tiles");
    const uint32_t sx_n = (uint32_t)((c.dw + STRIP_PX - 1) / STRIP_PX);
    const int ty = (int)(strip / sx_n), sx = (int)(strip % sx_n);
    const int px = sx * STRIP_PX + lane;
    const bool xin = px < c.dw;
    uint32_t D[TILE_PX];
#pragma unroll
    for (int r = 0; r < TILE_PX; ++r) {  // the eight row reads are independent
        const int py = ty * TILE_PX + r;
        D[r] = xin && py < c.dh ? depth[(size_t)py * c.dw + px] : 0u;
    }
    uint32_t mn = 0xFFFFu, mx = 0u;
    const float ninf = __int_as_float(0xff800000);
#pragma unroll
    for (int r = 0; r < TILE_PX; ++r) {
        const int py = ty * TILE_PX + r;
        if (depth_m && xin && py < c.dh) depth_m[(size_t)py * c.dw + px] = D[r] ? (float)D[r] * 0.001f : ninf;
        mn = min(mn, D[r] ? D[r] : 0xFFFFu);
        mx = max(mx, D[r]);
    }
#pragma unroll
    for (int o = 1; o < TILE_PX; o <<= 1) {  // within each group of eight lanes
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int tx = sx * 4 + (lane >> 3);
    if ((lane & 7) == 0 && tx < c.tiles_x) tiles[ty * c.tiles_x + tx] = mn | (mx << 16);
}

__global__ void __launch_bounds__(TILES_THREADS) k_depth_tiles(FrameConst c, const uint16_t* __restrict__ depth,
                                                               uint32_t* __restrict__ tiles,
                                                               Counters* __restrict__ ctr,
                                                               float* __restrict__ depth_m) {
    chain_enter();
    const int lane = threadIdx.x & 31;
    const uint32_t strip = blockIdx.x * (TILES_THREADS / 32) + (threadIdx.x >> 5);
    if (strip < depth_strips(c)) depth_strip(c, depth, tiles, depth_m, strip, lane);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // fold the previous frame's geometry-side counters into the running
        // totals (the colour side is folded by the geometry kernel, so this
        // kernel may run while the previous frame's colour work finishes)
        ctr->tot_geo_updated += ctr->geo_updated;
        ctr->tot_geo_bricks += ctr->n_geo;
        ctr->tot_vis_bricks += ctr->n_vis;
        ctr->tot_geo_changed += ctr->n_geo_changed;
        ctr->n_geo_changed = 0;
        ctr->frames += 1ull;
        ctr->n_geo = ctr->n_vis = 0;
        ctr->geo_next = 0;
        ctr->geo_updated = 0ull;
    }
}

dim3 depth_tiles_grid(const FrameConst& c) {
    return dim3((depth_strips(c) + TILES_THREADS / 32 - 1) / (TILES_THREADS / 32));
}

// ------------------------------------------------------------ bricks ----
// One thread per geometry brick.  A brick is "visible" unless one of these
// proves that no voxel (geometry or colour) inside it can be updated:
//   - its padded extent projects outside the depth image;
//   - every depth tile under that projection is invalid (D = 0);
//   - it lies more than max(mu, sigma) + margin beyond the farthest depth
//     under its projection (the sdf < -mu skip, and Eq. 7 for colour).
// A visible brick needs no geometry work when every voxel it holds would be
// left unchanged: it lies in front of the nearest depth by more than mu and
// either free-space updates are off or the brick is saturated free space
// (all F = 1, all w = max_weight), where (1 * w + 1) / (w + 1) = 1.  The
// visible list (the colour candidates) also drops bricks lying in front of
// the nearest depth by more than sigma + margin.
// Image-plane footprint of the axis-aligned box [lo, hi] (world): the bounds
// of its 8 projected corners, its camera-z range, whether some corner is (near)
// behind the camera (straddle: the footprint is then the whole image) and
// whether every corner is behind it (behind: no point of the box projects).
struct Footprint {
    float umin, umax, vmin, vmax, zmin, zmax;
    bool straddle, behind;
};

__device__ __forceinline__ Footprint box_footprint(const FrameConst& c, const float lo[3], const float hi[3]) {
    Footprint f{FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX, false, true};
    // camera and homogeneous image coordinates are affine in the corner, so
    // the corners are the lo corner plus sums of three edge vectors
    float X0[3], dX[3][3], h0[3], dh[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        X0[r] = c.R[3 * r] * lo[0] + c.R[3 * r + 1] * lo[1] + c.R[3 * r + 2] * lo[2] + c.t[r];
#pragma unroll
        for (int a = 0; a < 3; ++a) dX[r][a] = c.R[3 * r + a] * (hi[a] - lo[a]);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        h0[r] = c.Kd[3 * r] * X0[0] + c.Kd[3 * r + 1] * X0[1] + c.Kd[3 * r + 2] * X0[2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            dh[r][a] = c.Kd[3 * r] * dX[0][a] + c.Kd[3 * r + 1] * dX[1][a] + c.Kd[3 * r + 2] * dX[2][a];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float Z = X0[2], xh = h0[0], yh = h0[1], zh = h0[2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if ((k >> a) & 1) {
                Z += dX[2][a];
                xh += dh[0][a];
                yh += dh[1][a];
                zh += dh[2][a];
            }
        f.zmin = fminf(f.zmin, Z);
        f.zmax = fmaxf(f.zmax, Z);
        f.behind = f.behind && zh < -1e-5f;  // margin over the rounding of the corner sums
        if (zh <= 1e-4f) { f.straddle = true; continue; }
        const float rz = __frcp_rn(zh);
        const float u = xh * rz, v = yh * rz;
        f.umin = fminf(f.umin, u); f.umax = fmaxf(f.umax, u);
        f.vmin = fminf(f.vmin, v); f.vmax = fmaxf(f.vmax, v);
    }
    return f;
}

// The footprint lies beyond the image by more than the padding (2 pixels,
// far above the error of the approximate quotients), or the box is wholly
// behind the camera: no voxel in it projects into the image.
__device__ __forceinline__ bool outside_image(const FrameConst& c, const Footprint& f) {
    if (f.behind) return true;
    return !f.straddle && (f.umax < -2.0f || f.vmax < -2.0f || f.umin > (float)c.dw + 1.0f ||
                           f.vmin > (float)c.dh + 1.0f);
}

// Quick conservative test for a pinhole depth camera: the ball around the
// padded brick (centre p, radius r) lies wholly behind the camera, or wholly
// in front and beyond the image: then no voxel of the brick projects into
// the image.  Over the ball X' is within X +- r, Y' within Y +- r and Z' within
// Z +- r > 0, so u = fx X' / Z' + cx is bounded by its values at those ends.
__device__ __forceinline__ bool ball_outside_image(const FrameConst& c, const float p[3], float r) {
    const float X = c.R[0] * p[0] + c.R[1] * p[1] + c.R[2] * p[2] + c.t[0];
    const float Y = c.R[3] * p[0] + c.R[4] * p[1] + c.R[5] * p[2] + c.t[1];
    const float Z = c.R[6] * p[0] + c.R[7] * p[1] + c.R[8] * p[2] + c.t[2];
    if (Z + r < 0.0f) return true;
    if (!(Z - r > 1e-3f)) return false;  // may straddle the camera plane: decide with the box
    const float i0 = __frcp_rn(Z - r), i1 = __frcp_rn(Z + r);
    const float xa = X - r, xb = X + r, ya = Y - r, yb = Y + r;
    const float u0 = c.Kd[0] * xa * i0, u1 = c.Kd[0] * xa * i1, u2 = c.Kd[0] * xb * i0, u3 = c.Kd[0] * xb * i1;
    const float v0 = c.Kd[4] * ya * i0, v1 = c.Kd[4] * ya * i1, v2 = c.Kd[4] * yb * i0, v3 = c.Kd[4] * yb * i1;
    const float umin = fminf(fminf(u0, u1), fminf(u2, u3)) + c.Kd[2], umax = fmaxf(fmaxf(u0, u1), fmaxf(u2, u3)) + c.Kd[2];
    const float vmin = fminf(fminf(v0, v1), fminf(v2, v3)) + c.Kd[5], vmax = fmaxf(fmaxf(v0, v1), fmaxf(v2, v3)) + c.Kd[5];
    // one pixel more than the box test's padding covers the rounding here
    return umax < -3.0f || vmax < -3.0f || umin > (float)c.dw + 2.0f || vmin > (float)c.dh + 2.0f;
}

__device__ __forceinline__ void brick_flags(const FrameConst& c, const BrickSummary* __restrict__ summ,
                                            const uint32_t* __restrict__ tiles, uint32_t b, bool in, bool& geo,
                                            bool& vis, bool& inner) {
    vis = in;
    geo = in;
    inner = false;
    if (in && c.culling) {
        int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        if (c.kd_pinhole) {
            const float p[3] = {c.origin[0] + (float)(bx * BRICK + BRICK / 2) * c.s_g,
                                c.origin[1] + (float)(by * BRICK + BRICK / 2) * c.s_g,
                                c.origin[2] + (float)(bz * BRICK + BRICK / 2 + c.zoff_g) * c.s_g};
            // half-diagonal of the padded brick (4.5 voxels per axis) with 0.1 % and 10 um to spare
            const float r = fmaf(7.8e-3f, c.s_g, 1e-5f) + 4.5f * 1.7320508f * c.s_g;
            if (ball_outside_image(c, p, r)) {
                vis = geo = false;
                return;
            }
        }
        const BrickSummary s = summ[b];  // read early: its latency overlaps the footprint and tile reads
        float lo[3], hi[3];
        const int v0[3] = {bx * BRICK, by * BRICK, bz * BRICK + c.zoff_g};  // global index of the brick's first voxel
        for (int a = 0; a < 3; ++a) {
            lo[a] = c.origin[a] + ((float)v0[a] - 0.5f) * c.s_g;
            hi[a] = c.origin[a] + ((float)(v0[a] + BRICK) + 0.5f) * c.s_g;
        }
        const Footprint fp = box_footprint(c, lo, hi);
        float umin = fp.umin, umax = fp.umax, vmin = fp.vmin, vmax = fp.vmax;
        const float zmin = fp.zmin, zmax = fp.zmax;
        const bool straddle = fp.straddle;
        int px0 = 0, px1 = c.dw - 1, py0 = 0, py1 = c.dh - 1;
        if (outside_image(c, fp)) {
            vis = false;
        } else if (!straddle) {
            // every corner is in front of the camera and the footprint lies
            // more than a pixel inside the image: every voxel of the brick is
            // in front and projects into the image (the geometry update then
            // skips its per-voxel image tests)
            inner = umin > 1.0f && vmin > 1.0f && umax < (float)c.dw - 2.0f && vmax < (float)c.dh - 2.0f;
            // clamp before converting so the integer bounds cannot overflow
            umin = fmaxf(umin, -4.0f); umax = fminf(umax, (float)c.dw + 4.0f);
            vmin = fmaxf(vmin, -4.0f); vmax = fminf(vmax, (float)c.dh + 4.0f);
            px0 = max(0, (int)floorf(umin) - 2); px1 = min(c.dw - 1, (int)ceilf(umax) + 2);
            py0 = max(0, (int)floorf(vmin) - 2); py1 = min(c.dh - 1, (int)ceilf(vmax) + 2);
        }
        uint32_t dmin = 0xFFFFu, dmax = 0u;
        if (vis) {
            int tx0 = px0 / TILE_PX, tx1 = px1 / TILE_PX, ty0 = py0 / TILE_PX, ty1 = py1 / TILE_PX;
            if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 256 && tx1 - tx0 < 16) {
                // the reads of a tile row are independent: issue them together,
                // eight at a time
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int x0 = tx0; x0 <= tx1; x0 += 8) {
                        const uint32_t* row = tiles + ty * c.tiles_x + x0;
                        uint32_t tv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) tv[i] = x0 + i <= tx1 ? __ldg(row + i) : 0xFFFFu;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            dmin = min(dmin, tv[i] & 0xFFFFu);
                            dmax = max(dmax, tv[i] >> 16);
                        }
                    }
            } else {
                dmin = 1u;
                dmax = 0xFFFFu;
            }
            if (dmax == 0u) vis = false;                                   // no measurement under it
            else if (zmin > (float)dmax * 0.001f + c.cull_behind) vis = false;  // hidden behind every surface
        }
        // the geometry update skips sdf < -mu, so mu (not max(mu, sigma)) bounds it
        geo = vis && !(zmin > (float)dmax * 0.001f + c.mu + 2e-3f);
        if (vis) {
            bool sat = c.free_space == 0 || (s.fmin == 1.0f && s.wmin == (uint32_t)c.max_weight);
            if (sat && zmax < (float)dmin * 0.001f - c.mu - 2e-3f) geo = false;
            // colour: Eq. 7 needs |Z - d| <= sigma (pinhole K_c: the back-projected
            // point has Z = d), so a brick wholly nearer than the nearest depth
            // minus sigma holds no colour voxel that can pass
            if (c.kdi_pinhole && zmax < (float)dmin * 0.001f - c.cull_behind) vis = false;
        }
    }
}

// Append the flagged values of a whole block to two lists with one atomic per
// list per block (all threads of the block call it): thousands of warps
// finishing together would otherwise queue on the two counters.
template <int NT>
__device__ __forceinline__ void block_append2(bool p0, bool p1, uint32_t value0, uint32_t value1, uint32_t* ctr0,
                                              uint32_t* list0, uint32_t* ctr1, uint32_t* list1) {
    constexpr int NW = NT / 32;
    __shared__ uint32_t off[2][NW + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
    if (lane == 0) {
        off[0][wid] = __popc(m0);
        off[1][wid] = __popc(m1);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        uint32_t tot = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t n = off[threadIdx.x][w];
            off[threadIdx.x][w] = tot;
            tot += n;
        }
        off[threadIdx.x][NW] = tot ? atomicAdd(threadIdx.x ? ctr1 : ctr0, tot) : 0u;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    if (p0) list0[off[0][NW] + off[0][wid] + __popc(m0 & lt)] = value0;
    if (p1) list1[off[1][NW] + off[1][wid] + __popc(m1 & lt)] = value1;
    __syncthreads();  // off is reused by the block's next call
}

// The same for three lists, the third filled from its end down: its k-th
// value goes to list2_end[-1 - k].
template <int NT>
__device__ __forceinline__ void block_append3(bool p0, bool p1, bool p2, uint32_t value0, uint32_t value1,
                                              uint32_t value2, uint32_t* ctr0, uint32_t* list0, uint32_t* ctr1,
                                              uint32_t* list1, uint32_t* ctr2, uint32_t* list2_end) {
    constexpr int NW = NT / 32;
    __shared__ uint32_t off[3][NW + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned m[3] = {__ballot_sync(0xffffffffu, p0), __ballot_sync(0xffffffffu, p1),
                           __ballot_sync(0xffffffffu, p2)};
    if (lane == 0) {
        off[0][wid] = __popc(m[0]);
        off[1][wid] = __popc(m[1]);
        off[2][wid] = __popc(m[2]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        uint32_t tot = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t n = off[threadIdx.x][w];
            off[threadIdx.x][w] = tot;
            tot += n;
        }
        uint32_t* ctr = threadIdx.x == 0 ? ctr0 : (threadIdx.x == 1 ? ctr1 : ctr2);
        off[threadIdx.x][NW] = tot ? atomicAdd(ctr, tot) : 0u;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    if (p0) list0[off[0][NW] + off[0][wid] + __popc(m[0] & lt)] = value0;
    if (p1) list1[off[1][NW] + off[1][wid] + __popc(m[1] & lt)] = value1;
    if (p2) list2_end[-1 - (int64_t)(off[2][NW] + off[2][wid] + __popc(m[2] & lt))] = value2;
    __syncthreads();  // off is reused by the block's next call
}

// Add per-warp counts (the same value in every lane of a warp) to up to three
// global counters with one atomic per counter per block (all threads of the
// block call it): the warps of a balanced kernel end together, and one atomic
// per warp on one address would queue behind each other.
template <int NT, typename T0, typename T1 = uint32_t, typename T2 = uint32_t>
__device__ __forceinline__ void block_add(uint32_t v0, T0* d0, uint32_t v1 = 0u, T1* d1 = nullptr, uint32_t v2 = 0u,
                                          T2* d2 = nullptr) {
    constexpr int NW = NT / 32;
    __shared__ uint32_t part[3][NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        part[0][wid] = v0;
        part[1][wid] = v1;
        part[2][wid] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        uint32_t sum = 0;
        for (int w = 0; w < NW; ++w) sum += part[threadIdx.x][w];
        if (sum) {
            if (threadIdx.x == 0) atomicAdd(d0, (T0)sum);
            else if (threadIdx.x == 1 && d1) atomicAdd(d1, (T1)sum);
            else if (threadIdx.x == 2 && d2) atomicAdd(d2, (T2)sum);
        }
    }
}

// Geometry work-list entry: the brick's coordinates (10 bits per axis; the
// volume has at most 4096 voxels = 512 bricks per axis) and, in bit 31, the
// interior flag (the brick projects wholly into the image).
constexpr uint32_t GEO_INNER = 0x80000000u;
__device__ __forceinline__ uint32_t geo_entry(const FrameConst& c, uint32_t b, bool inner) {
    const uint32_t nb0 = (uint32_t)c.nb[0], nb1 = (uint32_t)c.nb[1];
    const uint32_t bx = b % nb0, r = b / nb0, by = r % nb1, bz = r / nb1;
    return bx | by << 10 | bz << 20 | (inner ? GEO_INNER : 0u);
}
struct BrickAt {
    uint32_t b;
    int bx, by, bz;
};
__device__ __forceinline__ BrickAt geo_brick(const FrameConst& c, uint32_t e) {
    BrickAt a;
    a.bx = (int)(e & 1023u);
    a.by = (int)((e >> 10) & 1023u);
    a.bz = (int)((e >> 20) & 1023u);
    a.b = (uint32_t)a.bx + (uint32_t)c.nb[0] * ((uint32_t)a.by + (uint32_t)c.nb[1] * (uint32_t)a.bz);
    return a;
}

constexpr int BRICK_THREADS = 64;  // small blocks: they fit beside the band kernel's blocks on an SM

// Brick culling: the geometry work list and the visible list; for the fused
// frame also each brick's state byte (listed, visible) and a fresh ready queue.
__global__ void __launch_bounds__(BRICK_THREADS) k_bricks(FrameConst c, const BrickSummary* __restrict__ summ,
                                                const uint32_t* __restrict__ tiles, Counters* __restrict__ ctr,
                                                uint32_t* __restrict__ geo_list, uint32_t* __restrict__ vis_list,
                                                uint8_t* __restrict__ bstate, FuseSync* __restrict__ fsync) {
    chain_enter();
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    bool geo, vis, inner;
    brick_flags(c, summ, tiles, b, b < nbt, geo, vis, inner);
    if (c.fused) {
        if (b < nbt) bstate[b] = (uint8_t)((geo ? 1u : 0u) | (vis ? 2u : 0u));
        if (b == 0) {
            fsync->head = 0u;
            fsync->tail = 0u;
        }
    }
    // geometry list entries carry the interior flag in bit 31
    block_append2<BRICK_THREADS>(geo, vis, geo_entry(c, b, inner), b, &ctr->n_geo, geo_list, &ctr->n_vis,
                                 vis_list);
}

// ---------------------------------------------------------- geometry ----
// TSDF update (the KinectFusion step the paper inherits, Section III):
//   D = depth at the nearest pixel of the voxel centre (Eq. 6); D = 0 skipped
//   sdf = D * 0.001 - Z; sdf < -mu skipped; (free space off: sdf > mu skipped)
//   t = min(1, sdf * (1/mu)); F <- fmaf(F, w, t) / (w + 1); w <- min(w+1, max_w)
// One warp per brick.  Lane l owns the four float4 groups q = l + 32 j
// (j = 0..3) of the brick: voxels 4q..4q+3, i.e. x in {0..3} or {4..7},
// y = (l >> 1) & 7, z = (l >> 4) + 2 j.  Each group of the warp is 512
// contiguous bytes of F and 128 of w.  The warp then writes the brick summary
// (min/max F over observed voxels, min w, band flags).

// Two voxels per instruction: the sm_100 paired binary32 operations
// (__ffma2_rn, __fmul2_rn, __fadd2_rn, __fadd2_rd) round each component
// exactly as the scalar operation does, so a pair of voxels follows the
// per-voxel definition bit for bit while the arithmetic issues half as often.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Nearest depth pixel of a pair of camera points (Eq. 6: xh = fmaf(K0, X,
// K2 Z) for a pinhole K, u = xh (1/zh), pixel floor(u + 1/2)).  The floor is
// taken as (u + 1/2) + 2^23 rounded toward minus infinity, whose bits are
// 0x4B000000 + floor(u + 1/2) for 0 <= u + 1/2 < 2^23 and fall outside the
// image test for any other value (negative, huge or infinite), so the
// integer test 0 <= floor < W is the float test 0 <= u + 1/2 < W.  The pixel
// index iv W + iu is then (bits of v) W + (bits of u) - 0x4B000000 (W + 1),
// modulo 2^32.  INNER: the caller knows every point lies in front of the
// camera and inside the image.  Otherwise a point outside the image gets
// pixel 0 and ok = false.
template <bool PINHOLE, bool INNER>
__device__ __forceinline__ void depth_pixels(const FrameConst& c, float2 X, float2 Y, float2 Z, uint32_t pix[2],
                                             bool ok[2]) {
    float2 xh, yh, zh;
    if (PINHOLE) {
        xh = __ffma2_rn(f2(c.Kd[0]), X, __fmul2_rn(f2(c.Kd[2]), Z));
        yh = __ffma2_rn(f2(c.Kd[4]), Y, __fmul2_rn(f2(c.Kd[5]), Z));
        zh = Z;
    } else {
        xh = __ffma2_rn(f2(c.Kd[0]), X, __ffma2_rn(f2(c.Kd[1]), Y, __fmul2_rn(f2(c.Kd[2]), Z)));
        yh = __ffma2_rn(f2(c.Kd[3]), X, __ffma2_rn(f2(c.Kd[4]), Y, __fmul2_rn(f2(c.Kd[5]), Z)));
        zh = __ffma2_rn(f2(c.Kd[6]), X, __ffma2_rn(f2(c.Kd[7]), Y, __fmul2_rn(f2(c.Kd[8]), Z)));
    }
    const float2 rz = rcp2_rn(zh);
    const float2 bu = __fadd2_rd(__fadd2_rn(__fmul2_rn(xh, rz), f2(0.5f)), f2(8388608.0f));
    const float2 bv = __fadd2_rd(__fadd2_rn(__fmul2_rn(yh, rz), f2(0.5f)), f2(8388608.0f));
    const uint32_t u0 = __float_as_uint(bu.x), u1 = __float_as_uint(bu.y);
    const uint32_t v0 = __float_as_uint(bv.x), v1 = __float_as_uint(bv.y);
    const uint32_t dw = (uint32_t)c.dw;
    pix[0] = v0 * dw + u0 - c.pix_bias;
    pix[1] = v1 * dw + u1 - c.pix_bias;
    if (INNER) {
        ok[0] = ok[1] = true;
    } else {
        ok[0] = zh.x > 0.0f && u0 - 0x4B000000u < dw && v0 - 0x4B000000u < (uint32_t)c.dh;
        ok[1] = zh.y > 0.0f && u1 - 0x4B000000u < dw && v1 - 0x4B000000u < (uint32_t)c.dh;
        if (!ok[0]) pix[0] = 0u;
        if (!ok[1]) pix[1] = 0u;
    }
}

// Any byte of v zero (the classic word trick: a borrow reaches the byte's top
// bit only from a zero byte).
__device__ __forceinline__ bool any_zero_byte(uint32_t v) { return ((v - 0x01010101u) & ~v & 0x80808080u) != 0u; }

// 0x01 in each byte of v that is zero, 0x00 in the others (exact per byte:
// (b & 0x7F) + 0x7F carries into bit 7 iff b & 0x7F != 0, and never out of the byte).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t v) {
    return ~(((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v | 0x7F7F7F7Fu) >> 7;
}

// Minimum / maximum of a float over the warp (sm_100 warp reduction; no NaN
// reaches it here).
__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// Depth sources of the update.  The frame's depth image in mm (D = 0: no
// measurement), or the same in metres as the depth-tile kernel writes it
// (RN(D * 0.001), -inf where D = 0): a -inf depth gives sdf = -inf < -mu,
// which the update skips as it skips D = 0.
struct DepthMm {
    const uint16_t* __restrict__ p;
};
struct DepthM {
    const float* __restrict__ p;
};

// TSDF update of geometry brick `at` by one warp (lane = lane index) from its
// F and w already loaded (f, wv: this lane's four groups); writes the changed
// groups and the brick summary.  Adds the number of updated voxels to count
// and 1 to changed if any voxel changed.
//   D = depth at the nearest pixel of the voxel centre (Eq. 6); D = 0 skipped
//   sdf = D * 0.001 - Z; sdf < -mu skipped; (free space off: sdf > mu skipped)
//   t = min(1, sdf * (1/mu)); F <- fmaf(F, w, t) / (w + 1); w <- min(w+1, max_w)
// One warp per brick.  Lane l owns the four float4 groups q = l + 32 j
// (j = 0..3) of the brick: voxels 4q..4q+3, i.e. x in {0..3} or {4..7},
// y = (l >> 1) & 7, z = (l >> 4) + 2 j.  Each group of the warp is 512
// contiguous bytes of F and 128 of w.
template <bool PINHOLE, bool FREE_SPACE, bool ALIGNED, bool INNER, typename Depth>
__device__ __forceinline__ void geometry_update(const FrameConst& c, const Volumes& vol, Depth depth,
                                                const BrickAt& at, int lane, const float4 (&f)[4],
                                                const uint32_t (&wv)[4], uint32_t& count, uint32_t& changed) {
    constexpr bool METRES = std::is_same<Depth, DepthM>::value;
    const int lx = (lane & 1) * 4, ly = (lane >> 1) & 7, lz = lane >> 4;
    float* Fb = vol.F + (size_t)at.b * BRICK_VOX + lane * 4;
    uint8_t* Wb = vol.W + (size_t)at.b * BRICK_VOX + lane * 4;
    const int gx0 = at.bx * BRICK + lx, gy = at.by * BRICK + ly;
    const bool yin = gy < c.ng[1];
    const float py = fmaf((float)gy + 0.5f, c.s_g, c.origin[1]);
    // voxel centres (index + 1/2) s + origin; the integer + 1/2 sums below are exact
    const float gxf = (float)gx0;
    const float2 pxp[2] = {make_float2(fmaf(gxf + 0.5f, c.s_g, c.origin[0]), fmaf(gxf + 1.5f, c.s_g, c.origin[0])),
                           make_float2(fmaf(gxf + 2.5f, c.s_g, c.origin[0]), fmaf(gxf + 3.5f, c.s_g, c.origin[0]))};
    const float gzf = (float)(at.bz * BRICK + lz + c.zoff_g) + 0.5f;  // centre at the global index
    const uint32_t maxw = (uint32_t)c.max_weight, maxw4 = maxw * 0x01010101u;
    // min / max of F over this lane's observed voxels: all of them, and those
    // on the brick faces (band flags): this lane's x face is its voxel i = 0
    // (lx = 0, the -x face) or i = 3 (lx = 4, +x), its z face its group j = 0
    // (lz = 0, -z) or j = 3 (lz = 1, +z).  An unobserved voxel enters as NaN,
    // which fminf / fmaxf pass over.
    const float qnan = __int_as_float(0x7fffffff);
    float fmn = FLT_MAX, fmx = -FLT_MAX, mn_xf = FLT_MAX, mx_xf = -FLT_MAX, mn_zf = FLT_MAX, mx_zf = -FLT_MAX;
    bool unobserved = false, below_cap = false;  // after the update, over this lane's in-volume voxels
    uint32_t upd = 0;                            // updated voxels of this lane, bit 4 j + i
    // The groups in two halves of two: first the pixels and depth reads of a
    // half's eight voxels, then their updates, so that the eight reads are in
    // flight together (a depth the update may not use reads as -inf, which
    // the sdf gate rejects).  All sixteen at once need more than the 64
    // registers that eight blocks per SM allow.
    constexpr int GS = 2;  // groups per half
#pragma unroll
    for (int j0 = 0; j0 < 4; j0 += GS) {
        float2 dd[GS][2];
#pragma unroll
        for (int jj = 0; jj < GS; ++jj) {
            const int j = j0 + jj;
            const int gz = at.bz * BRICK + lz + 2 * j;
            const bool zin = yin && gz < c.ng[2];
            const float pz = fmaf(gzf + (float)(2 * j), c.s_g, c.origin[2]);
            const float2 B0 = f2(fmaf(c.R[1], py, fmaf(c.R[2], pz, c.t[0])));
            const float2 B1 = f2(fmaf(c.R[4], py, fmaf(c.R[5], pz, c.t[1])));
            const float2 B2 = f2(fmaf(c.R[7], py, fmaf(c.R[8], pz, c.t[2])));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 X = __ffma2_rn(f2(c.R[0]), pxp[h], B0);
                const float2 Y = __ffma2_rn(f2(c.R[3]), pxp[h], B1);
                const float2 Z = __ffma2_rn(f2(c.R[6]), pxp[h], B2);
                uint32_t pix[2];
                bool ok[2], has[2];  // has: a depth the update may use
                depth_pixels<PINHOLE, INNER>(c, X, Y, Z, pix, ok);
#pragma unroll
                for (int k = 0; k < 2; ++k)  // ALIGNED: dims are multiples of 8
                    has[k] = ok[k] && (ALIGNED || (zin && gx0 + 2 * h + k < c.ng[0]));
                float2 d;
                if constexpr (METRES) {  // the metres image holds -inf where D = 0
                    d = make_float2(__ldg(depth.p + pix[0]), __ldg(depth.p + pix[1]));
                } else {
                    // RN(D * 0.001) as fmaf(2^23 + D, 0.001, -2^23 * 0.001): the product is exact
                    // inside the fma and 2^23 * 0.001f is a power-of-two scaling, so one rounding
                    const uint32_t D0 = __ldg(depth.p + pix[0]), D1 = __ldg(depth.p + pix[1]);
                    d = __ffma2_rn(make_float2(__uint_as_float(0x4B000000u | D0), __uint_as_float(0x4B000000u | D1)),
                                   f2(0.001f), f2(-8388608.0f * 0.001f));
                    has[0] = has[0] && D0 != 0u;
                    has[1] = has[1] && D1 != 0u;
                }
                if (!(INNER && ALIGNED && METRES)) {
                    d.x = has[0] ? d.x : -INFINITY;
                    d.y = has[1] ? d.y : -INFINITY;
                }
                dd[jj][h] = d;
            }
        }
#pragma unroll
        for (int jj = 0; jj < GS; ++jj) {
            const int j = j0 + jj;
            const int gz = at.bz * BRICK + lz + 2 * j;
            const bool zin = yin && gz < c.ng[2];
            const float pz = fmaf(gzf + (float)(2 * j), c.s_g, c.origin[2]);
            const float2 B2 = f2(fmaf(c.R[7], py, fmaf(c.R[8], pz, c.t[2])));
            const float fin[4] = {f[j].x, f[j].y, f[j].z, f[j].w};
            float fv[4], fo[4];
            const uint32_t w_old = wv[j];
            uint32_t upm = 0, inside = 0xFFFFFFFFu;
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // voxel pair i = 2h, 2h + 1
                const float2 Z = __ffma2_rn(f2(c.R[6]), pxp[h], B2);  // as in the first pass
                bool valid[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int i = 2 * h + k;
                    valid[k] = ALIGNED || (zin && gx0 + i < c.ng[0]);
                    if (!valid[k]) inside &= ~(0xFFu << (8 * i));
                }
                const float2 d = dd[jj][h];
                const float2 sdf = __ffma2_rn(Z, f2(-1.0f), d);  // d - Z, rounded once
                const float2 tq = __fmul2_rn(sdf, f2(c.inv_mu));
                const float2 t = make_float2(fminf(1.0f, tq.x), fminf(1.0f, tq.y));
                // w as binary32 from its byte: the bits 0x4B0000ww are 2^23 + w
                const uint32_t wb0 = __byte_perm(w_old, 0x4B000000u, 0x7440u + 2 * h);
                const uint32_t wb1 = __byte_perm(w_old, 0x4B000000u, 0x7441u + 2 * h);
                const float2 wbf = make_float2(__uint_as_float(wb0), __uint_as_float(wb1));
                const float2 wf = __fadd2_rn(wbf, f2(-8388608.0f));               // w, exact
                const float2 nb = __ffma2_rn(wbf, f2(-1.0f), f2(8388607.0f));     // -(w + 1), exact
                const float2 y = rcp2_rn(__fadd2_rn(wbf, f2(-8388607.0f)));  // RN(1 / (w + 1)), w + 1 exact
                // F <- fmaf(F, w, t) / (w + 1), the quotient by div_by_weight's steps
                const float2 a = __ffma2_rn(make_float2(fin[2 * h], fin[2 * h + 1]), wf, t);
                const float2 q = __fmul2_rn(a, y);
                const float2 r = __ffma2_rn(nb, q, a);
                const float2 fn = __ffma2_rn(r, y, q);
                const float sd[2] = {sdf.x, sdf.y}, fnew[2] = {fn.x, fn.y};
                const uint32_t wb[2] = {wb0, wb1};
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int i = 2 * h + k;
                    const bool up = !(sd[k] < -c.mu) && (FREE_SPACE || !(sd[k] > c.mu));
                    fv[i] = up ? fnew[k] : fin[i];
                    upm |= up ? 1u << i : 0u;
                    fo[i] = (up || wb[k] != 0x4B000000u) && valid[k] ? fv[i] : qnan;  // observed after the update
                }
            }
            // w <- min(w + 1, max_weight): +1 in the updated bytes that are below the cap
            const uint32_t upb = (upm * 0x00204081u) & 0x01010101u;  // bit i of upm -> byte i
            const uint32_t wn = w_old + (upb & ~zero_bytes(w_old ^ maxw4));
            // in-volume voxels only: a byte outside the volume reads as observed and at the cap
            const uint32_t wq = ALIGNED ? wn : (wn & inside) | (maxw4 & ~inside);
            unobserved = unobserved || any_zero_byte(wq);
            below_cap = below_cap || wq != maxw4;
            const float gmn = fminf(fminf(fo[0], fo[1]), fminf(fo[2], fo[3]));
            const float gmx = fmaxf(fmaxf(fo[0], fo[1]), fmaxf(fo[2], fo[3]));
            fmn = fminf(fmn, gmn);
            fmx = fmaxf(fmx, gmx);
            // this lane's x-face voxel of the group, and its z-face group
            const float fx = lx == 0 ? fo[0] : fo[3];
            mn_xf = fminf(mn_xf, fx);
            mx_xf = fmaxf(mx_xf, fx);
            if ((j == 0 && lz == 0) || (j == 3 && lz == 1)) {
                mn_zf = gmn;
                mx_zf = gmx;
            }
            upd |= upm << (4 * j);
            if (upm) {
                *reinterpret_cast<float4*>(Fb + 128 * j) = make_float4(fv[0], fv[1], fv[2], fv[3]);
                *reinterpret_cast<uint32_t*>(Wb + 128 * j) = wn;
            }
        }
    }
    count += __popc(upd);
    // bricks where nothing changed keep their summary
    if (!__any_sync(0xffffffffu, upd != 0u)) return;
    ++changed;
    // band flags (see BrickSummary): this lane's voxels sit at x = lx + i,
    // y = ly, z = lz + 2 j, so it holds the -x face when lx = 0, +x when
    // lx = 4, -y / +y when ly = 0 / 7, -z when lz = 0 and +z when lz = 1
    const float lo_thr = c.band + CELL_EPS, hi_thr = -c.band - CELL_EPS;
    auto lohi = [&](bool on, float mn, float mx) -> uint32_t {
        return on ? (mn <= lo_thr ? 1u : 0u) | (mx >= hi_thr ? 2u : 0u) : 0u;
    };
    const uint32_t xf = lohi(true, mn_xf, mx_xf), zf = lohi(true, mn_zf, mx_zf);
    uint32_t bflags = lohi(true, fmn, fmx) | (lx == 0 ? xf << 2 : xf << 4) | lohi(ly == 0, fmn, fmx) << 6 |
                      lohi(ly == 7, fmn, fmx) << 8 | (lz == 0 ? zf << 10 : zf << 12);
    fmn = warp_min(fmn);
    fmx = warp_max(fmx);
    unobserved = __any_sync(0xffffffffu, unobserved);
    below_cap = __any_sync(0xffffffffu, below_cap);
    bflags = __reduce_or_sync(0xffffffffu, bflags);
    if (lane == 0) {
        BrickSummary sm;
        sm.fmin = fmn == FLT_MAX ? __int_as_float(0x7f800000) : fmn;
        sm.fmax = fmx == -FLT_MAX ? __int_as_float(0xff800000) : fmx;
        sm.wmin = unobserved ? 0u : (below_cap ? maxw - 1u : maxw);
        sm.flags = bflags;
        vol.summ[at.b] = sm;
    }
}

// The same with F and w read from the volume: all four groups' loads are
// issued before the first update (the stores of a group could otherwise hold
// back the next group's loads).
template <bool PINHOLE, bool FREE_SPACE, bool ALIGNED = false, bool INNER = false, typename Depth>
__device__ __forceinline__ void geometry_brick(const FrameConst& c, const Volumes& vol, Depth depth,
                                               const BrickAt& at, int lane, uint32_t& count, uint32_t& changed) {
    const float* Fb = vol.F + (size_t)at.b * BRICK_VOX + lane * 4;
    const uint8_t* Wb = vol.W + (size_t)at.b * BRICK_VOX + lane * 4;
    float4 f[4];
    uint32_t wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[j] = *reinterpret_cast<const float4*>(Fb + 128 * j);
        wv[j] = *reinterpret_cast<const uint32_t*>(Wb + 128 * j);
    }
    geometry_update<PINHOLE, FREE_SPACE, ALIGNED, INNER>(c, vol, depth, at, lane, f, wv, count, changed);
}

template <bool PINHOLE, bool FREE_SPACE, bool ALIGNED>
__global__ void __launch_bounds__(GEO_THREADS, 8) k_geometry(FrameConst c, Volumes vol, const float* __restrict__ depth_m,
                                                          Counters* __restrict__ ctr,
                                                          const uint32_t* __restrict__ list) {
    chain_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // fold the previous frame's colour-side counters into the running totals
        ctr->tot_col_updated += ctr->col_updated;
        ctr->tot_col_bricks += ctr->n_col + ctr->n_col_light;
        ctr->tot_cells += ctr->n_cells;
        ctr->tot_col_active += ctr->n_col_active;
        ctr->n_col = ctr->col_next = ctr->n_col_light = 0;
        ctr->n_cells = ctr->n_vox = ctr->n_col_active = 0;
        ctr->col_updated = 0ull;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = ctr->n_geo;
    const DepthM depth{depth_m};
    uint32_t count = 0, changed = 0;
    // the list is taken from its end: the colour kernels that follow walk
    // their lists from the front, whose bricks are then the ones this kernel
    // wrote last (measured: 1 % off the frame)
    for (uint32_t item = warp; item < n; item += nwarps) {
        const uint32_t e = list[n - 1u - item];
        const BrickAt at = geo_brick(c, e);
        if (e & GEO_INNER)  // the brick projects wholly into the image: no per-voxel image tests
            geometry_brick<PINHOLE, FREE_SPACE, ALIGNED, true>(c, vol, depth, at, lane, count, changed);
        else
            geometry_brick<PINHOLE, FREE_SPACE, ALIGNED, false>(c, vol, depth, at, lane, count, changed);
    }
    block_add<GEO_THREADS>(__reduce_add_sync(0xffffffffu, count), &ctr->geo_updated, changed, &ctr->n_geo_changed);
}

// Launch with programmatic stream serialization (the kernel begins with
// chain_enter()), so its launch overlaps the drain of the kernel before it.
template <typename... Params, typename... Args>
cudaError_t launch_chained(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// Launch the k_geometry instance for this frame's camera model, free-space
// mode and volume shape (every dimension a multiple of 8: no bounds tests).
// It reads the depth in metres that this frame's k_depth_tiles wrote.
cudaError_t launch_k_geometry(const FrameConst& c, const Volumes& v, const Scratch& s, int grid, cudaStream_t stream) {
    const bool aligned = c.ng[0] % BRICK == 0 && c.ng[1] % BRICK == 0 && c.ng[2] % BRICK == 0;
    const int key = (c.kd_pinhole ? 4 : 0) | (c.free_space ? 2 : 0) | (aligned ? 1 : 0);
    switch (key) {
#define TSDF_GEO_CASE(k, P, F, A) \
    case k: return launch_chained(k_geometry<P, F, A>, dim3(grid), dim3(GEO_THREADS), 0, stream, c, v, s.depth_m, \
                                  s.ctr, s.geo_list);
        TSDF_GEO_CASE(0, false, false, false)
        TSDF_GEO_CASE(1, false, false, true)
        TSDF_GEO_CASE(2, false, true, false)
        TSDF_GEO_CASE(3, false, true, true)
        TSDF_GEO_CASE(4, true, false, false)
        TSDF_GEO_CASE(5, true, false, true)
        TSDF_GEO_CASE(6, true, true, false)
        TSDF_GEO_CASE(7, true, true, true)
#undef TSDF_GEO_CASE
    }
    return cudaGetLastError();
}

// ------------------------------------------------------- colour list ----
// A visible geometry brick goes to the colour list when some trilinear cell
// of the colour voxels it owns can have corners on both sides of the band:
// a brick owns the cells whose lower corner lies in it, so their corners lie
// in the brick and in the first voxel layers of its seven + neighbours
// (+x, +y, +z, the three edges and the corner between them), and the brick
// needs an observed voxel with F <= band + eps and one with F >= -band - eps
// among its own voxels and those layers.  A face neighbour contributes its
// touching face layer (its -x, -y or -z face); an edge or corner neighbour
// contributes only voxels on all of its touching faces, so the AND of those
// faces' flags is still a necessary condition.
// Colour-candidate test of a visible geometry brick (see above).
__device__ __forceinline__ bool colour_candidate(const FrameConst& c, const BrickSummary* __restrict__ summ,
                                                 uint32_t b) {
    if (!c.culling) return true;
    const int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
    uint32_t acc = summ[b].flags & 3u;
#pragma unroll
    for (int k = 1; k < 8; ++k) {  // no early exit: the reads are independent
        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
        const int x = bx + dx, y = by + dy, z = bz + dz;
        if (x >= c.nb[0] || y >= c.nb[1] || z >= c.nb[2]) continue;
        const uint32_t f = summ[((size_t)z * c.nb[1] + y) * c.nb[0] + x].flags;
        // the neighbour at +x touches with its -x face (bits 2-3), +y with -y (6-7), +z with -z (10-11)
        uint32_t m = 3u;
        if (dx) m &= f >> 2;
        if (dy) m &= f >> 6;
        if (dz) m &= f >> 10;
        acc |= m & 3u;
    }
    return acc == 3u;
}

constexpr int LIST_THREADS = 256;
constexpr uint8_t BUSY_CELLS = 32;  // active cells from which a candidate goes to the list's front

__global__ void __launch_bounds__(LIST_THREADS) k_colour_list(FrameConst c, const BrickSummary* __restrict__ summ,
                                                     Counters* __restrict__ ctr, const uint32_t* __restrict__ vis_list,
                                                     uint32_t* __restrict__ col_list,
                                                     const uint8_t* __restrict__ col_act) {
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    // The visible list and its length come from the brick culling, which had
    // finished before the geometry kernel this one follows could start, so
    // they are read before waiting for the geometry kernel (the summaries it
    // writes are read after).
    const uint32_t n = ctr->n_vis;
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t b_next = i0 < n ? vis_list[i0] : 0u;
    chain_enter();
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t b = b_next;
        const uint32_t in = i + gridDim.x * blockDim.x;
        b_next = in < n ? vis_list[in] : 0u;
        const bool act = i < n && colour_candidate(c, summ, b);
        // bricks with many active cells at their last band gate take the
        // longest: they go first, the others to the list's end
        const bool busy = act && col_act[b] >= BUSY_CELLS;
        block_append3<LIST_THREADS>(busy, false, act && !busy, b, b, b, &ctr->n_col, col_list, nullptr, nullptr,
                                    &ctr->n_col_light, col_list + nbt);
    }
}

// ------------------------------------------------------------ colour ----
// HD sample (Eq. 9): nearest pixel, or bilinear over the 2x2 neighbourhood
// (inside the image), rounded half-up.
__device__ __forceinline__ bool sample_rgb(const FrameConst& c, const uint8_t* __restrict__ rgb, float u, float v,
                                           uint32_t s[3]) {
    if (c.sample_mode == 0) {
        int iu, iv;
        if (!nearest_pixel(u, v, c.cw, c.ch, iu, iv)) return false;
        const uint8_t* px = rgb + ((size_t)iv * c.cw + iu) * 3;
        s[0] = __ldg(px);
        s[1] = __ldg(px + 1);
        s[2] = __ldg(px + 2);
        return true;
    }
    const float x0 = floorf(u), y0 = floorf(v);
    if (!(x0 >= 0.0f && x0 + 1.0f <= (float)(c.cw - 1) && y0 >= 0.0f && y0 + 1.0f <= (float)(c.ch - 1))) return false;
    const float ax = u - x0, ay = v - y0;
    const uint8_t* r0 = rgb + ((size_t)(int)y0 * c.cw + (int)x0) * 3;
    const uint8_t* r1 = r0 + (size_t)c.cw * 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p00 = (float)__ldg(r0 + k), p10 = (float)__ldg(r0 + 3 + k);
        const float p01 = (float)__ldg(r1 + k), p11 = (float)__ldg(r1 + 3 + k);
        const float top = fmaf(ax, p10 - p00, p00);
        const float bot = fmaf(ax, p11 - p01, p01);
        const float val = fmaf(ay, bot - top, top);
        s[k] = (uint32_t)floorf(val + 0.5f);
    }
    return true;
}

// Eq. 8-10 update (colour_mode 1); returns whether the voxel changed.
__device__ __forceinline__ bool paper_normal_update(const FrameConst& c, const uint16_t* __restrict__ depth, int iu,
                                                    int iv, float PdX, float PdY, float PdZ, float X, float Y, float Z,
                                                    uint32_t& vox, const uint32_t s[3]) {
    if (!(iu + 1 <= c.dw - 1 && iv + 1 <= c.dh - 1)) return false;
    const uint32_t D1 = __ldg(depth + (size_t)iv * c.dw + iu + 1);
    const uint32_t D2 = __ldg(depth + (size_t)(iv + 1) * c.dw + iu);
    if (D1 == 0u || D2 == 0u) return false;
    float X1, Y1, Z1, X2, Y2, Z2;
    back_project(c, iu + 1, iv, (float)D1 * 0.001f, X1, Y1, Z1);
    back_project(c, iu, iv + 1, (float)D2 * 0.001f, X2, Y2, Z2);
    const float a0 = X1 - PdX, a1 = Y1 - PdY, a2 = Z1 - PdZ;
    const float b0 = X2 - PdX, b1 = Y2 - PdY, b2 = Z2 - PdZ;
    const float n0 = fmaf(a1, b2, -(a2 * b1));
    const float n1 = fmaf(a2, b0, -(a0 * b2));
    const float n2 = fmaf(a0, b1, -(a1 * b0));
    const float nn = __fsqrt_rn(fmaf(n0, n0, fmaf(n1, n1, n2 * n2)));
    const float pn = __fsqrt_rn(fmaf(X, X, fmaf(Y, Y, Z * Z)));
    if (!(nn > 0.0f && pn > 0.0f)) return false;
    const float dot = fmaf(n0, X, fmaf(n1, Y, n2 * Z));
    const float Wc = __fdiv_rn(dot, nn * pn);
    if (!(Wc > 0.0f)) return false;
    uint32_t wq = (uint32_t)floorf(fmaf(Wc, 255.0f, 0.5f));
    if (wq > 255u) wq = 255u;
    const uint32_t wp = vox >> 24;
    if (!(5u * wq > 4u * wp)) return false;
    const uint32_t den = wp + wq;
    uint32_t out = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint32_t cc = (vox >> (8 * k)) & 0xFFu;
        out |= ((cc * wp + s[k] * wq + (den >> 1)) / den) << (8 * k);
    }
    const uint32_t wn = wp + (wq * (255u - wp) + 127u) / 255u;
    vox = out | (wn << 24);
    return true;
}

// Colour update of one colour voxel (Section IV.B) that has passed the
// trilinear band gate, given its indices k:
//   Eq. 5 -> Eq. 6 -> D > 0 -> Eq. 7 sigma gate -> Eq. 3-4 -> HD sample
//   -> Eq. 9 (integer, half-up) or Eq. 8-10.
// (The gates are independent predicates, so testing the band first changes
// nothing.)  Returns whether the voxel was updated.
__device__ __forceinline__ bool colour_after_band(const FrameConst& c, uint32_t* __restrict__ C,
                                                  const uint16_t* __restrict__ depth, const uint8_t* __restrict__ rgb,
                                                  int kx, int ky, int kz) {
    const float pwx = fmaf((float)kx + 0.5f, c.s_c, c.origin[0]);
    const float pwy = fmaf((float)ky + 0.5f, c.s_c, c.origin[1]);
    const float pwz = fmaf((float)(kz + c.zoff_c) + 0.5f, c.s_c, c.origin[2]);  // global index on a z-slab
    float X, Y, Z;
    rigid(c.R, c.t, pwx, pwy, pwz, X, Y, Z);
    float u, v;
    int iu, iv;
    if (!project(c.Kd, c.kd_pinhole, X, Y, Z, u, v)) return false;
    if (!nearest_pixel(u, v, c.dw, c.dh, iu, iv)) return false;
    const uint32_t D = __ldg(depth + (size_t)iv * c.dw + iu);
    if (D == 0u) return false;
    const float d = (float)D * 0.001f;
    float PdX, PdY, PdZ;
    back_project(c, iu, iv, d, PdX, PdY, PdZ);
    const float ex = X - PdX, ey = Y - PdY, ez = Z - PdZ;
    const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    if (dist2 > c.sigma2) return false;
    float Xh, Yh, Zh;
    rigid(c.Rc, c.tc, X, Y, Z, Xh, Yh, Zh);
    float uh, vh;
    if (!project(c.Kr, c.kr_pinhole, Xh, Yh, Zh, uh, vh)) return false;
    uint32_t smp[3];
    if (!sample_rgb(c, rgb, uh, vh, smp)) return false;
    const int64_t co = brick_offset(kx, ky, kz, c.ncb);
    uint32_t vox = C[co];
    if (c.colour_mode == 1) {
        if (!paper_normal_update(c, depth, iu, iv, PdX, PdY, PdZ, X, Y, Z, vox, smp)) return false;
    } else {
        const uint32_t w = vox >> 24;
        uint32_t out = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t cc = (vox >> (8 * k)) & 0xFFu;
            out |= ((cc * w + smp[k] + ((w + 1u) >> 1)) / (w + 1u)) << (8 * k);
        }
        const uint32_t wn = min(w + 1u, (uint32_t)c.max_weight);
        vox = out | (wn << 24);
    }
    C[co] = vox;
    return true;
}

// Band gate of the colour voxels a geometry brick owns (first colour
// kernel): those whose trilinear cell has its lower corner in the brick, so
// every owned cell lies between the brick's voxels 0..8 on each axis.  One
// warp per listed brick, taken with an atomic counter.  The warp
//   1. stages the brick's post-update geometry plus the first voxel layers of
//      its + neighbours (9^3 F and w: the brick as float4, the halo as 3
//      faces, 3 edges and 1 corner) in its shared-memory slot with three flag
//      bits per voxel: observed (w > 0), F <= band + eps, F >= -band - eps;
//      and tabulates, per axis, the owned colour indices' cells and fractions;
//   2. packs the flags into 9-bit row masks;
//   3. marks the 8^3 trilinear cells that can pass the band gate (all eight
//      corners observed, the corner range meets [-band, band]) as 8-bit masks
//      (AND / OR of four rows, then of neighbouring bits) and compacts them;
//   4. evaluates the trilinear TSDF (lerp along x, then y, then z) of every
//      colour voxel of a marked cell and records those with |F| <= band for
//      the colour-voxel kernel, through a shared staging buffer kept across
//      the warp's bricks (one atomic per flush of up to STAGE records).
//      Records that do not fit the global buffer are finished by the warp
//      itself (same arithmetic).
// The cell marks are conservative (eps bounds the trilinear rounding); the
// band gate itself is evaluated exactly as written.
constexpr int MAXK = 66;    // owned colour indices per axis (colour/geometry ratio <= 8)
constexpr int STAGE = 512;  // per-warp record staging entries (kept across a warp's bricks)

struct ColourSlot {  // one warp's shared-memory working set (~9 KB)
    float F[TILE_G3];
    // per tile row (z * 9 + y): bit x = observed, bit 9 + x = F <= band + eps,
    // bit 18 + x = F >= -band - eps
    uint32_t row[TILE_G * TILE_G];
    uint16_t cells[CELLS3];
    float frac[3][MAXK];
    uint8_t start[3][CELLS], end[3][CELLS];
    int32_t nbr[8];  // the brick and its + neighbours, (sz * 2 + sy) * 2 + sx; -1 outside the volume
    uint2 out[STAGE];
};

// Store one staged geometry voxel with its flags.
// Row-mask bits of one voxel (see ColourSlot::row), at x = 0.
__device__ __forceinline__ uint32_t voxel_bits(float f, uint32_t w, float lo_thr, float hi_thr) {
    return (w != 0u ? 1u : 0u) | (f <= lo_thr ? 1u << 9 : 0u) | (f >= hi_thr ? 1u << 18 : 0u);
}

// Store one staged geometry voxel and its row-mask bits.
__device__ __forceinline__ void stage(ColourSlot& S, int tx, int ty, int tz, float f, uint32_t w, float lo_thr,
                                      float hi_thr) {
    const int r = tz * TILE_G + ty;
    S.F[r * TILE_G + tx] = f;
    const uint32_t bits = voxel_bits(f, w, lo_thr, hi_thr) << tx;
    if (bits) atomicOr(&S.row[r], bits);
}

// Offset of tile voxel (tx, ty, tz) in the brick-major volume, or -1.  Tile
// coordinates 0..7 are the brick's locals 0..7, 8 is local 0 of the next brick.
__device__ __forceinline__ int64_t tile_offset(const ColourSlot& S, int tx, int ty, int tz) {
    const int sx = tx >> 3, sy = ty >> 3, sz = tz >> 3;
    const int nb = S.nbr[(sz * 2 + sy) * 2 + sx];
    if (nb < 0) return -1;
    return (int64_t)nb * BRICK_VOX + ((tz & 7) * BRICK + (ty & 7)) * BRICK + (tx & 7);
}

// The band kernel's overflow path, kept out of line: inlined, its registers
// and code weigh on the whole band kernel although it almost never runs.
__device__ __noinline__ bool colour_after_band_outlined(const FrameConst& c, uint32_t* __restrict__ C,
                                                        const uint16_t* __restrict__ depth,
                                                        const uint8_t* __restrict__ rgb, int kx, int ky, int kz) {
    return colour_after_band(c, C, depth, rgb, kx, ky, kz);
}

// Write n staged records to the global list from slot `base` on (warp-
// uniform); those beyond its capacity are finished here.  Returns the number
// of colour voxels updated here.
__device__ uint32_t write_records(const FrameConst& c, const Volumes& vol, const uint16_t* __restrict__ depth,
                                  const uint8_t* __restrict__ rgb, const Scratch& scr, const ColourSlot& S,
                                  uint32_t n, uint32_t base, int lane) {
    uint32_t done = 0;
    // the records that fit are copied in a loop of their own: with the rare
    // overflow call inside it, the copy loop cost the band kernel 15 %
    const uint32_t fit = base >= scr.vox_cap ? 0u : min(n, scr.vox_cap - base);
    for (uint32_t i = lane; i < fit; i += 32) scr.vox[base + i] = S.out[i];
    if (fit < n) {  // beyond the buffer
        if (c.record_mode) {
            if (lane == 0) atomicOr(scr.err, ERR_RECORD_OVERFLOW);  // recording has no fallback; the host reports it
        } else {
            for (uint32_t i = fit + lane; i < n; i += 32) {
                const uint2 r = S.out[i];
                if (colour_after_band_outlined(c, vol.C, depth, rgb, (int)(r.x & 0xFFFFu), (int)(r.x >> 16), (int)r.y))
                    ++done;
            }
        }
    }
    __syncwarp();
    return done;
}

// Claim slots for n staged records and write them.
__device__ uint32_t flush_records(const FrameConst& c, const Volumes& vol, const uint16_t* __restrict__ depth,
                                  const uint8_t* __restrict__ rgb, const Scratch& scr, const ColourSlot& S,
                                  uint32_t n, int lane) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&scr.ctr->n_vox, n);
    base = __shfl_sync(0xffffffffu, base, 0);
    return write_records(c, vol, depth, rgb, scr, S, n, base, lane);
}

// Band gate of the colour voxels owned by geometry brick b, by one warp with
// shared-memory slot S (steps 1-4 above).
// Records stay in S.out (nstage of them) across the warp's bricks: the caller
// flushes what is left (band_flush) when its bricks are done.
__device__ __forceinline__ void band_brick(const FrameConst& c, const Volumes& vol, const uint16_t* __restrict__ depth,
                                           const uint8_t* __restrict__ rgb, const Scratch& scr, ColourSlot& S,
                                           uint32_t b, int lane, uint32_t& count, uint32_t& n_active,
                                           uint32_t& n_cells, uint32_t& nstage) {
    const unsigned full = 0xffffffffu;
    const float lo_thr = c.band + CELL_EPS, hi_thr = -c.band - CELL_EPS;
    const int bb[3] = {(int)(b % c.nb[0]), (int)((b / c.nb[0]) % c.nb[1]), (int)(b / (c.nb[0] * c.nb[1]))};
    // owned colour ranges and per-cell spans from the per-axis tables
    int k0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) k0[a] = __ldg(vol.tab.k0[a] + bb[a]);
    // the first 32 owned indices' trilinear fractions per axis and the
    // per-axis cell summaries, read now so that their latency overlaps the
    // tile reads below (indices beyond 32, at ratios above 4: read in step 1c)
    int nk[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        nk[a] = __ldg(vol.tab.k0[a] + bb[a] + 1) - k0[a];
        fr[a] = lane < nk[a] ? __ldg(vol.tab.frac[a] + k0[a] + lane) : 0.0f;
    }
    const uint32_t xinfo = __ldg(vol.tab.info[0] + bb[0]);
    const uint32_t yinfo = __ldg(vol.tab.info[1] + bb[1]), zinfo = __ldg(vol.tab.info[2] + bb[2]);
    if (lane < 8) {
        const int x = bb[0] + (lane & 1), y = bb[1] + ((lane >> 1) & 1), z = bb[2] + (lane >> 2);
        S.nbr[lane] = (x < c.nb[0] && y < c.nb[1] && z < c.nb[2])
                          ? (int32_t)(((int64_t)z * c.nb[1] + y) * c.nb[0] + x)
                          : -1;
    }
    if (lane < 3 * CELLS) {
        const int a = lane / CELLS, cell = lane % CELLS;
        const int ba = a == 0 ? bb[0] : (a == 1 ? bb[1] : bb[2]);  // no dynamic indexing of bb
        const uint16_t* span = a == 0 ? vol.tab.span[0] : (a == 1 ? vol.tab.span[1] : vol.tab.span[2]);
        const uint16_t sp = __ldg(span + ba * CELLS + cell);
        S.start[a][cell] = (uint8_t)(sp & 0xFFu);
        S.end[a][cell] = (uint8_t)(sp >> 8);
    }
    for (int r = lane; r < TILE_G * TILE_G; r += 32) S.row[r] = 0u;
    __syncwarp();

    // 1a. centre brick: four float4 of F and four words of w per lane
    {
        const float* Fb = vol.F + (size_t)b * BRICK_VOX + lane * 4;
        const uint8_t* Wb = vol.W + (size_t)b * BRICK_VOX + lane * 4;
        float4 f[4];
        uint32_t wv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            f[j] = *reinterpret_cast<const float4*>(Fb + 128 * j);
            wv[j] = *reinterpret_cast<const uint32_t*>(Wb + 128 * j);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = lane + 32 * j;
            const int x0 = (q & 1) * 4, y = (q >> 1) & 7, z = q >> 4;
            const int r = z * TILE_G + y, i = r * TILE_G + x0;
            S.F[i] = f[j].x;
            S.F[i + 1] = f[j].y;
            S.F[i + 2] = f[j].z;
            S.F[i + 3] = f[j].w;
            const uint32_t bits = (voxel_bits(f[j].x, wv[j] & 0xFFu, lo_thr, hi_thr) |
                                   voxel_bits(f[j].y, (wv[j] >> 8) & 0xFFu, lo_thr, hi_thr) << 1 |
                                   voxel_bits(f[j].z, (wv[j] >> 16) & 0xFFu, lo_thr, hi_thr) << 2 |
                                   voxel_bits(f[j].w, wv[j] >> 24, lo_thr, hi_thr) << 3)
                                  << x0;
            if (bits) atomicOr(&S.row[r], bits);
        }
    }
    // 1b. halo, the next bricks' first layers: 3 faces x 64, 3 edges x 8, 1 corner = 217 voxels
    {
        int txs[7], tys[7], tzs[7];
#pragma unroll
        for (int i = 0; i < 6; ++i) {  // faces: i = 2 * axis + half
            const int axis = i >> 1, q = lane + 32 * (i & 1);
            const int a = q & 7, bq = q >> 3;
            txs[i] = axis == 0 ? BRICK : a;
            tys[i] = axis == 1 ? BRICK : (axis == 0 ? a : bq);
            tzs[i] = axis == 2 ? BRICK : bq;
        }
        {  // edges (lanes 0..23, along axis lane / 8) and the corner (lane 24)
            const int e = lane >> 3, m = lane & 7;
            txs[6] = e == 0 ? m : BRICK;
            tys[6] = e == 1 ? m : BRICK;
            tzs[6] = e == 2 ? m : BRICK;
        }
        float hf[7];
        uint32_t hw[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int64_t off = (i < 6 || lane < 25) ? tile_offset(S, txs[i], tys[i], tzs[i]) : -1;
            hf[i] = off >= 0 ? vol.F[off] : 0.0f;
            hw[i] = off >= 0 ? (uint32_t)vol.W[off] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 7; ++i)
            if (i < 6 || lane < 25) stage(S, txs[i], tys[i], tzs[i], hf[i], hw[i], lo_thr, hi_thr);
    }
    // 1c. trilinear fraction of each owned colour index, from the per-axis tables
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (lane < nk[a]) S.frac[a][lane] = fr[a];
        for (int j = lane + 32; j < nk[a]; j += 32) S.frac[a][j] = __ldg(vol.tab.frac[a] + k0[a] + j);
    }
    __syncwarp();

    // 3. active cells, compacted
    // cells along x that own colour indices, and the most indices of one cell per axis
    const uint32_t xmask = xinfo & 0xFFu;
    const int mx = (int)(xinfo >> 9), my = (int)(yinfo >> 9), mz = (int)(zinfo >> 9);
    uint32_t act[2];
    uint32_t total = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int yz = lane + 32 * r;
        act[r] = 0;
        if (yz < CELLS * CELLS) {
            const int cy = yz % CELLS, cz = yz / CELLS;
            if (S.end[1][cy] > S.start[1][cy] && S.end[2][cz] > S.start[2][cz]) {
                const int r00 = cz * TILE_G + cy;
                const uint32_t w00 = S.row[r00], w10 = S.row[r00 + 1], w01 = S.row[r00 + TILE_G],
                               w11 = S.row[r00 + TILE_G + 1];
                uint32_t o = w00 & w10 & w01 & w11 & 0x1FFu;
                o &= o >> 1;
                uint32_t a = o & xmask;
                if (c.culling) {
                    const uint32_t any = w00 | w10 | w01 | w11;
                    const uint32_t l = (any >> 9) & 0x1FFu, h = (any >> 18) & 0x1FFu;
                    a &= (l | (l >> 1)) & (h | (h >> 1));
                }
                act[r] = a & 0xFFu;
            }
        }
        total += __popc(act[r]);
    }
    uint32_t incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t nact = __shfl_sync(full, incl, 31);
    if (lane == 0 && scr.col_act) scr.col_act[b] = (uint8_t)min(nact, 255u);  // orders the next frame's list
    if (nact == 0) return;  // no colour voxel of this brick can pass the band gate
    ++n_active;
    n_cells += nact;
    uint32_t pos = incl - total;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        uint32_t a = act[r];
        const int yz = lane + 32 * r;
        while (a) {
            const int cx = __ffs(a) - 1;
            a &= a - 1;
            S.cells[pos++] = (uint16_t)(yz * CELLS + cx);
        }
    }
    __syncwarp();

    // 4. band gate of the colour voxels of the active cells, one lane per
    // cell: the x-lerps of an index jx serve every (jy, jz) of the cell and
    // the y-lerps of (jx, jy) every jz (the same operations as one lerp chain
    // per voxel).
    if (mx <= 2 && my <= 2 && mz <= 2) {
        // At most two owned indices per axis (colour/geometry ratio up to 2):
        // a lane evaluates its cell's (at most eight) colour voxels into a
        // pass mask, bit 4 ix + 2 iy + iz, and one prefix sum over the warp
        // places the batch's records.
        for (uint32_t cb = 0; cb < nact; cb += 32) {
            uint32_t mask = 0;
            uint32_t jx0 = 0, jy0 = 0, jz0 = 0;
            if (cb + lane < nact) {
                const uint32_t cellid = S.cells[cb + lane];
                const int cx = cellid % CELLS, cy = (cellid / CELLS) % CELLS, cz = cellid / (CELLS * CELLS);
                const int sx = S.start[0][cx], sy = S.start[1][cy], sz = S.start[2][cz];
                const int nx = S.end[0][cx] - sx, ny = S.end[1][cy] - sy, nz = S.end[2][cz] - sz;
                const int o = (cz * TILE_G + cy) * TILE_G + cx;
                const float q000 = S.F[o], q100 = S.F[o + 1], q010 = S.F[o + TILE_G], q110 = S.F[o + TILE_G + 1];
                const float q001 = S.F[o + TILE_G * TILE_G], q101 = S.F[o + TILE_G * TILE_G + 1];
                const float q011 = S.F[o + TILE_G * TILE_G + TILE_G], q111 = S.F[o + TILE_G * TILE_G + TILE_G + 1];
                const float fx[2] = {S.frac[0][sx], S.frac[0][nx > 1 ? sx + 1 : sx]};
                const float fy[2] = {S.frac[1][sy], S.frac[1][ny > 1 ? sy + 1 : sy]};
                const float fz[2] = {S.frac[2][sz], S.frac[2][nz > 1 ? sz + 1 : sz]};
#pragma unroll
                for (int ix = 0; ix < 2; ++ix) {
                    const float c00 = lerp(q000, q100, fx[ix]), c10 = lerp(q010, q110, fx[ix]);
                    const float c01 = lerp(q001, q101, fx[ix]), c11 = lerp(q011, q111, fx[ix]);
#pragma unroll
                    for (int iy = 0; iy < 2; ++iy) {
                        const float c0 = lerp(c00, c10, fy[iy]), c1 = lerp(c01, c11, fy[iy]);
#pragma unroll
                        for (int iz = 0; iz < 2; ++iz)
                            if (fabsf(lerp(c0, c1, fz[iz])) <= c.band) mask |= 1u << (4 * ix + 2 * iy + iz);
                    }
                }
                // only the indices the cell owns
                const uint32_t own = nx > 0 && ny > 0 && nz > 0
                                         ? (nx > 1 ? 0xFFu : 0x0Fu) & (ny > 1 ? 0xFFu : 0x33u) & (nz > 1 ? 0xFFu : 0x55u)
                                         : 0u;
                mask &= own;
                jx0 = (uint32_t)(k0[0] + sx);
                jy0 = (uint32_t)(k0[1] + sy);
                jz0 = (uint32_t)(k0[2] + sz);
            }
            const uint32_t cnt = __popc(mask);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t total = __shfl_sync(full, incl, 31);
            if (nstage + total > STAGE) {  // a batch holds at most 256 records
                __syncwarp();
                count += flush_records(c, vol, depth, rgb, scr, S, nstage, lane);
                nstage = 0;
            }
            uint32_t pos = nstage + incl - cnt;
            while (mask) {
                const int bit = __ffs(mask) - 1;
                mask &= mask - 1u;
                S.out[pos++] = make_uint2((jx0 + (uint32_t)(bit >> 2)) | ((jy0 + (uint32_t)((bit >> 1) & 1)) << 16),
                                          jz0 + (uint32_t)(bit & 1));
            }
            nstage += total;
        }
        return;
    }
    // The general case: loops run to the warp-wide most indices per axis so
    // the record ballots stay uniform.
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    for (uint32_t cb = 0; cb < nact; cb += 32) {
        const bool live = cb + lane < nact;
        int sx = 0, ex = 0, sy = 0, ey = 0, sz = 0, ez = 0;
        float q000 = 0.0f, q100 = 0.0f, q010 = 0.0f, q110 = 0.0f, q001 = 0.0f, q101 = 0.0f, q011 = 0.0f,
              q111 = 0.0f;
        if (live) {
            const uint32_t cellid = S.cells[cb + lane];
            const int cx = cellid % CELLS, cy = (cellid / CELLS) % CELLS, cz = cellid / (CELLS * CELLS);
            sx = S.start[0][cx];
            ex = S.end[0][cx];
            sy = S.start[1][cy];
            ey = S.end[1][cy];
            sz = S.start[2][cz];
            ez = S.end[2][cz];
            const int o = (cz * TILE_G + cy) * TILE_G + cx;
            q000 = S.F[o];
            q100 = S.F[o + 1];
            q010 = S.F[o + TILE_G];
            q110 = S.F[o + TILE_G + 1];
            q001 = S.F[o + TILE_G * TILE_G];
            q101 = S.F[o + TILE_G * TILE_G + 1];
            q011 = S.F[o + TILE_G * TILE_G + TILE_G];
            q111 = S.F[o + TILE_G * TILE_G + TILE_G + 1];
        }
        for (int ix = 0; ix < mx; ++ix) {
            const int jx = sx + ix;
            const bool vx = live && jx < ex;
            const float fx = S.frac[0][vx ? jx : 0];
            const float c00 = lerp(q000, q100, fx), c10 = lerp(q010, q110, fx);
            const float c01 = lerp(q001, q101, fx), c11 = lerp(q011, q111, fx);
            for (int iy = 0; iy < my; ++iy) {
                const int jy = sy + iy;
                const bool vy = vx && jy < ey;
                const float fy = S.frac[1][vy ? jy : 0];
                const float c0 = lerp(c00, c10, fy), c1 = lerp(c01, c11, fy);
                for (int iz = 0; iz < mz; ++iz) {
                    const int jz = sz + iz;
                    const bool vz = vy && jz < ez;
                    const float fz = S.frac[2][vz ? jz : 0];
                    const bool pass = vz && fabsf(lerp(c0, c1, fz)) <= c.band;
                    const uint32_t m = __ballot_sync(full, pass);
                    if (pass)
                        S.out[nstage + __popc(m & lanemask_lt)] =
                            make_uint2((uint32_t)(k0[0] + jx) | ((uint32_t)(k0[1] + jy) << 16), (uint32_t)(k0[2] + jz));
                    nstage += __popc(m);
                    if (nstage > STAGE - 32) {
                        __syncwarp();
                        count += flush_records(c, vol, depth, rgb, scr, S, nstage, lane);
                        nstage = 0;
                    }
                }
            }
        }
    }
}

// The records a warp still holds in S.out.
__device__ __forceinline__ void band_flush(const FrameConst& c, const Volumes& vol, const uint16_t* __restrict__ depth,
                                           const uint8_t* __restrict__ rgb, const Scratch& scr, const ColourSlot& S,
                                           int lane, uint32_t& count, uint32_t& nstage) {
    __syncwarp();
    if (nstage) count += flush_records(c, vol, depth, rgb, scr, S, nstage, lane);
    nstage = 0;
}

__global__ void __launch_bounds__(COL_THREADS, 5) k_colour_band(FrameConst c, Volumes vol,
                                                                const uint16_t* __restrict__ depth,
                                                                const uint8_t* __restrict__ rgb, Scratch scr) {
    chain_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColourSlot& S = reinterpret_cast<ColourSlot*>(smem_raw)[threadIdx.x >> 5];
    Counters* __restrict__ ctr = scr.ctr;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    // the list's front part (bricks busy at their last band gate), then its
    // part filled from the buffer's end
    const uint32_t nh = ctr->n_col, n = nh + ctr->n_col_light;
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    uint32_t count = 0, n_active = 0, n_cells = 0, nstage = 0;
    // a warp's first item is its index in the grid, the later ones are
    // claimed from the counter (offset by the warp count), each while the
    // previous item is processed
    const uint32_t nwarps = gridDim.x * (COL_THREADS / 32);
    uint32_t next = blockIdx.x * (COL_THREADS / 32) + (threadIdx.x >> 5);
    for (;;) {
        const uint32_t item = __shfl_sync(full, next, 0);
        if (item >= n) break;
        if (lane == 0) next = nwarps + atomicAdd(&ctr->col_next, 1u);
        const uint32_t b = item < nh ? scr.col_list[item] : scr.col_list[nbt - 1u - (item - nh)];
        band_brick(c, vol, depth, rgb, scr, S, b, lane, count, n_active, n_cells, nstage);
        __syncwarp();
    }
    band_flush(c, vol, depth, rgb, scr, S, lane, count, nstage);
    // n_active and n_cells are the same in every lane
    block_add<COL_THREADS>(__reduce_add_sync(full, count), &ctr->col_updated, n_active, &ctr->n_col_active, n_cells,
                           &ctr->n_cells);
}

// Colour voxels that passed the band gate (second colour kernel): one thread
// per record, so the work is balanced however the surface is spread over
// bricks.
__global__ void __launch_bounds__(256) k_colour_voxels(FrameConst c, Volumes vol, const uint16_t* __restrict__ depth,
                                                       const uint8_t* __restrict__ rgb, Scratch scr) {
    chain_enter();
    Counters* __restrict__ ctr = scr.ctr;
    const uint32_t nv = min(ctr->n_vox, scr.vox_cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t count = 0;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint2 r = i < nv ? scr.vox[i] : make_uint2(0u, 0u);
    for (; i < nv; i += stride) {  // the next record is read while this one is updated
        const uint2 rn = i + stride < nv ? scr.vox[i + stride] : make_uint2(0u, 0u);
        if (colour_after_band(c, vol.C, depth, rgb, (int)(r.x & 0xFFFFu), (int)(r.x >> 16), (int)r.y)) ++count;
        r = rn;
    }
    block_add<256>(__reduce_add_sync(0xffffffffu, count), &ctr->col_updated);
}

// ------------------------------------------------------- fused frame ----
// The frame's geometry update, colour-candidate test and band gate in one
// persistent launch (the colour voxels follow in k_colour_voxels).  A visible
// brick's colour work reads the updated geometry of itself and its seven +
// neighbours, so it may start once every listed brick there has been updated:
// k_need counts those per visible brick; each warp that finishes a brick's
// geometry decrements the counts of the visible bricks that read it (itself
// and its seven - neighbours), and the warp that brings a count to zero
// pushes that brick on a ready queue.  Warps take at most one ready
// brick after each of their own geometry bricks (so the colour work runs
// beside the geometry), then, with their geometry done, the remaining ones.
// Only that last part waits, and only for bricks that the geometry still
// running will release; each wait is bounded (FUSE_WAIT_NS of %globaltimer or
// FUSE_WAIT_SPINS polls), after which the warp records ERR_WAIT_TIMEOUT in the
// handle's error word and stops.  Every block is resident (the grid is the
// occupancy times the SM count).
constexpr unsigned long long FUSE_WAIT_NS = 1000000000ull;  // 1 s
constexpr unsigned FUSE_WAIT_SPINS = 1u << 26;

__device__ __forceinline__ unsigned long long fuse_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Push brick b on this frame's ready queue (entries are tagged with the frame).
__device__ __forceinline__ void fuse_push(const FrameConst& c, const Scratch& scr, uint32_t b) {
    const uint32_t slot = atomicAdd(&scr.fsync->tail, 1u);
    const unsigned long long v = (unsigned long long)c.frame_tag << 32 | b;
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(scr.ready + slot), "l"(v) : "memory");
}

// Wait (bounded) until this frame's colour-side counters are reset and queue
// entry `slot` is written; b = its brick (all lanes).  Lane 0 polls with
// plain loads and a growing sleep, then one fence orders the warp's later
// reads after what it saw (acquire); false when the wait gave up.
__device__ __forceinline__ bool fuse_take(const FrameConst& c, const Scratch& scr, uint32_t slot, uint32_t& b,
                                          int lane) {
    uint32_t got = 0, v_lo = 0;
    if (lane == 0) {
        const volatile unsigned long long* p = scr.ready + slot;
        const volatile unsigned int* open = &scr.fsync->open;
        const unsigned long long t0 = fuse_ns();
        unsigned sleep = 32;
        for (unsigned spins = 0;; ++spins) {
            const unsigned long long v = *p;
            if ((uint32_t)(v >> 32) == c.frame_tag && *open == c.frame_tag) {
                v_lo = (uint32_t)v;
                got = 1;
                break;
            }
            if ((spins & 15u) == 15u && (fuse_ns() - t0 > FUSE_WAIT_NS || spins > FUSE_WAIT_SPINS)) break;
            __nanosleep(sleep);
            if (sleep < 1024) sleep *= 2;
        }
        if (got) __threadfence();
    }
    __syncwarp();
    got = __shfl_sync(0xffffffffu, got, 0);
    b = __shfl_sync(0xffffffffu, v_lo, 0);
    return got != 0;
}

// Visible bricks: count the listed bricks among themselves and their seven +
// neighbours; a brick with none is ready at once.  Test injection
// (FuseSync::stall): the first visible brick gets one count that no warp
// will release, so a wait for it runs out.
__global__ void __launch_bounds__(256) k_need(FrameConst c, Scratch scr) {
    chain_enter();
    const uint32_t n = scr.ctr->n_vis;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t b = scr.vis_list[i];
        const int bx = (int)(b % (uint32_t)c.nb[0]), by = (int)((b / (uint32_t)c.nb[0]) % (uint32_t)c.nb[1]),
                  bz = (int)(b / ((uint32_t)c.nb[0] * (uint32_t)c.nb[1]));
        uint32_t cnt = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {  // itself and its + neighbours: the geometry its colour work reads
            const int x = bx + (k & 1), y = by + ((k >> 1) & 1), z = bz + (k >> 2);
            if (x < c.nb[0] && y < c.nb[1] && z < c.nb[2])
                cnt += scr.bstate[((size_t)z * c.nb[1] + y) * c.nb[0] + x] & 1u;
        }
        if (i == 0 && *(volatile unsigned*)&scr.fsync->stall) {
            scr.fsync->stall = 0u;
            ++cnt;
        }
        scr.need[b] = cnt;
        if (cnt == 0u) fuse_push(c, scr, b);
    }
}

// colour_candidate with one lane per neighbour (lane 0: the brick itself).
__device__ __forceinline__ bool colour_candidate_warp(const FrameConst& c, const BrickSummary* __restrict__ summ,
                                                      uint32_t b, int lane) {
    if (!c.culling) return true;
    const int bx = (int)(b % (uint32_t)c.nb[0]), by = (int)((b / (uint32_t)c.nb[0]) % (uint32_t)c.nb[1]),
              bz = (int)(b / ((uint32_t)c.nb[0] * (uint32_t)c.nb[1]));
    uint32_t m = 0;
    if (lane < 8) {
        const int dx = lane & 1, dy = (lane >> 1) & 1, dz = lane >> 2;
        const int x = bx + dx, y = by + dy, z = bz + dz;
        if (x < c.nb[0] && y < c.nb[1] && z < c.nb[2]) {
            const uint32_t f = summ[((size_t)z * c.nb[1] + y) * c.nb[0] + x].flags;
            m = 3u;
            if (lane == 0) m &= f;
            if (dx) m &= f >> 2;
            if (dy) m &= f >> 6;
            if (dz) m &= f >> 10;
            m &= 3u;
        }
    }
    return __reduce_or_sync(0xffffffffu, m) == 3u;
}

// After a warp's geometry update of brick `at`: release its visible
// neighbours.  Each lane with one first fences (its F, w and summary stores,
// and through the warp barrier the other lanes', before its decrement).
__device__ __forceinline__ void fuse_release(const FrameConst& c, const Scratch& scr, const BrickAt& at, int lane) {
    __syncwarp();
    if (lane < 8) {  // the bricks whose colour work reads this one: itself and its - neighbours
        const int x = at.bx - (lane & 1), y = at.by - ((lane >> 1) & 1), z = at.bz - (lane >> 2);
        if (x >= 0 && y >= 0 && z >= 0) {
            const uint32_t nb = (uint32_t)(((size_t)z * c.nb[1] + y) * c.nb[0] + x);
            if (scr.bstate[nb] & 2u) {
                __threadfence();
                if (atomicSub(&scr.need[nb], 1u) == 1u) {
                    __threadfence();  // the other releases of nb happened before this one
                    fuse_push(c, scr, nb);
                }
            }
        }
    }
}

// The colour work of one ready visible brick.
__device__ __forceinline__ void fuse_colour(const FrameConst& c, const Volumes& vol, const uint16_t* __restrict__ depth,
                                            const uint8_t* __restrict__ rgb, const Scratch& scr, ColourSlot& S,
                                            uint32_t b, int lane, uint32_t& count, uint32_t& n_active,
                                            uint32_t& n_cells, uint32_t& n_cand, uint32_t& nstage) {
    if (!colour_candidate_warp(c, vol.summ, b, lane)) return;
    ++n_cand;
    band_brick(c, vol, depth, rgb, scr, S, b, lane, count, n_active, n_cells, nstage);
    __syncwarp();
}

template <bool FREE_SPACE, bool ALIGNED>
__global__ void __launch_bounds__(COL_THREADS, 5) k_fused(FrameConst c, Volumes vol, const uint16_t* __restrict__ depth,
                                                         const uint8_t* __restrict__ rgb, Scratch scr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColourSlot& S = reinterpret_cast<ColourSlot*>(smem_raw)[threadIdx.x >> 5];
    chain_enter();
    const unsigned full = 0xffffffffu;
    Counters* __restrict__ ctr = scr.ctr;
    FuseSync* __restrict__ fs = scr.fsync;
    if (threadIdx.x == 0 && atomicExch(&fs->claim, c.frame_tag) != c.frame_tag) {
        // the first block: fold the previous frame's colour-side counters into
        // the running totals, then let the colour work start
        ctr->tot_col_updated += ctr->col_updated;
        ctr->tot_col_bricks += ctr->n_col + ctr->n_col_light;
        ctr->tot_cells += ctr->n_cells;
        ctr->tot_col_active += ctr->n_col_active;
        ctr->n_col = ctr->col_next = ctr->n_col_light = 0;
        ctr->n_cells = ctr->n_vox = ctr->n_col_active = 0;
        ctr->col_updated = 0ull;
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&fs->open), "r"(c.frame_tag) : "memory");
    }
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = ctr->n_geo, nv = ctr->n_vis;
    const DepthM dm{scr.depth_m};
    uint32_t gcount = 0, changed = 0, count = 0, n_active = 0, n_cells = 0, n_cand = 0, nstage = 0;
    bool ok = true;
    // own geometry bricks, in list order (about z order: the bricks whose
    // neighbourhoods are complete follow the front), one ready colour brick
    // after each when the queue holds one
    for (uint32_t item = warp; item < n; item += nwarps) {
        const uint32_t e = scr.geo_list[item];
        const BrickAt at = geo_brick(c, e);
        if (e & GEO_INNER)
            geometry_brick<true, FREE_SPACE, ALIGNED, true>(c, vol, dm, at, lane, gcount, changed);
        else
            geometry_brick<true, FREE_SPACE, ALIGNED, false>(c, vol, dm, at, lane, gcount, changed);
        fuse_release(c, scr, at, lane);
        uint32_t slot = 0xFFFFFFFFu;
        if (lane == 0) {
            const uint32_t h = *(volatile unsigned*)&fs->head, t = *(volatile unsigned*)&fs->tail;
            if (h < t && *(volatile unsigned*)&fs->open == c.frame_tag && atomicCAS(&fs->head, h, h + 1u) == h)
                slot = h;
        }
        slot = __shfl_sync(full, slot, 0);
        if (slot != 0xFFFFFFFFu) {
            uint32_t b;
            if (!fuse_take(c, scr, slot, b, lane)) {
                ok = false;
                break;
            }
            fuse_colour(c, vol, depth, rgb, scr, S, b, lane, count, n_active, n_cells, n_cand, nstage);
        }
    }
    // the remaining ready bricks
    while (ok) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(&fs->head, 1u);
        slot = __shfl_sync(full, slot, 0);
        if (slot >= nv) break;
        uint32_t b;
        if (!fuse_take(c, scr, slot, b, lane)) {
            ok = false;
            break;
        }
        fuse_colour(c, vol, depth, rgb, scr, S, b, lane, count, n_active, n_cells, n_cand, nstage);
    }
    band_flush(c, vol, depth, rgb, scr, S, lane, count, nstage);
    if (!ok && lane == 0) atomicOr(scr.err, ERR_WAIT_TIMEOUT);
    gcount = __reduce_add_sync(full, gcount);
    count = __reduce_add_sync(full, count);
    if (lane == 0) {  // changed, n_active, n_cells and n_cand are the same in every lane
        if (gcount) atomicAdd(&ctr->geo_updated, (unsigned long long)gcount);
        if (changed) atomicAdd(&ctr->n_geo_changed, changed);
        if (count) atomicAdd(&ctr->col_updated, (unsigned long long)count);
        if (n_active) atomicAdd(&ctr->n_col_active, n_active);
        if (n_cells) atomicAdd(&ctr->n_cells, n_cells);
        if (n_cand) atomicAdd(&ctr->n_col, n_cand);
    }
}

// ------------------------------------------ caller-owned geometry volume ----
// Culling for the allocation-free geometry entry point: the frustum, empty
// footprint and hidden-behind tests of k_bricks, without the saturated
// free-space skip (that needs per-brick summaries, which this path does not
// keep).  Appends to the geometry work list only.
__global__ void __launch_bounds__(256) k_bricks_static(FrameConst c, const uint32_t* __restrict__ tiles,
                                                       Counters* __restrict__ ctr, uint32_t* __restrict__ geo_list) {
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    bool vis = b < nbt;
    if (vis && c.culling) {
        int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        float lo[3], hi[3];
        int bc[3] = {bx, by, bz};
        for (int a = 0; a < 3; ++a) {
            lo[a] = c.origin[a] + ((float)(bc[a] * BRICK) - 0.5f) * c.s_g;
            hi[a] = c.origin[a] + ((float)(bc[a] * BRICK + BRICK) + 0.5f) * c.s_g;
        }
        float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX, zmin = FLT_MAX;
        bool straddle = false;
        for (int k = 0; k < 8; ++k) {
            float x = (k & 1) ? hi[0] : lo[0], y = (k & 2) ? hi[1] : lo[1], z = (k & 4) ? hi[2] : lo[2];
            float X = c.R[0] * x + c.R[1] * y + c.R[2] * z + c.t[0];
            float Y = c.R[3] * x + c.R[4] * y + c.R[5] * z + c.t[1];
            float Z = c.R[6] * x + c.R[7] * y + c.R[8] * z + c.t[2];
            float xh = c.Kd[0] * X + c.Kd[1] * Y + c.Kd[2] * Z;
            float yh = c.Kd[3] * X + c.Kd[4] * Y + c.Kd[5] * Z;
            float zh = c.Kd[6] * X + c.Kd[7] * Y + c.Kd[8] * Z;
            zmin = fminf(zmin, Z);
            if (zh <= 1e-4f) { straddle = true; continue; }
            float u = xh / zh, v = yh / zh;
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
        }
        int px0 = 0, px1 = c.dw - 1, py0 = 0, py1 = c.dh - 1;
        if (!straddle) {
            if (umax < -2.0f || vmax < -2.0f || umin > (float)c.dw + 1.0f || vmin > (float)c.dh + 1.0f) {
                vis = false;
            } else {
                umin = fmaxf(umin, -4.0f); umax = fminf(umax, (float)c.dw + 4.0f);
                vmin = fmaxf(vmin, -4.0f); vmax = fminf(vmax, (float)c.dh + 4.0f);
                px0 = max(0, (int)floorf(umin) - 2); px1 = min(c.dw - 1, (int)ceilf(umax) + 2);
                py0 = max(0, (int)floorf(vmin) - 2); py1 = min(c.dh - 1, (int)ceilf(vmax) + 2);
            }
        }
        if (vis) {
            uint32_t dmax = 0u;
            int tx0 = px0 / TILE_PX, tx1 = px1 / TILE_PX, ty0 = py0 / TILE_PX, ty1 = py1 / TILE_PX;
            if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 256) {
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx) dmax = max(dmax, tiles[ty * c.tiles_x + tx] >> 16);
            } else {
                dmax = 0xFFFFu;
            }
            if (dmax == 0u) vis = false;
            else if (zmin > (float)dmax * 0.001f + c.cull_behind) vis = false;
        }
    }
    append(vis, b, &ctr->n_geo, geo_list);
}

// TSDF update of a caller-owned volume in linear x-fastest layout: the same
// per-voxel arithmetic as k_geometry (one warp per 8^3 brick of the work
// list, lane l owning x in {0..3} or {4..7}, y = (l >> 1) & 7,
// z = (l >> 4) + 2 j), with scalar loads and stores of the linear arrays and
// no brick summary.
template <bool PINHOLE, bool FREE_SPACE>
__global__ void __launch_bounds__(GEO_THREADS, 7) k_geometry_linear(FrameConst c, float* __restrict__ F,
                                                                 uint8_t* __restrict__ W,
                                                                 const uint16_t* __restrict__ depth,
                                                                 Counters* __restrict__ ctr,
                                                                 const uint32_t* __restrict__ list) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = ctr->n_geo;
    const int lx = (lane & 1) * 4, ly = (lane >> 1) & 7, lz = lane >> 4;
    uint32_t count = 0;
    for (uint32_t item = warp; item < n; item += nwarps) {
        const uint32_t b = list[item];
        const int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        const int gy = by * BRICK + ly;
        const float py = fmaf((float)gy + 0.5f, c.s_g, c.origin[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gz = bz * BRICK + lz + 2 * j;
            const float pz = fmaf((float)gz + 0.5f, c.s_g, c.origin[2]);
            const float B0 = fmaf(c.R[1], py, fmaf(c.R[2], pz, c.t[0]));
            const float B1 = fmaf(c.R[4], py, fmaf(c.R[5], pz, c.t[1]));
            const float B2 = fmaf(c.R[7], py, fmaf(c.R[8], pz, c.t[2]));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gx = bx * BRICK + lx + i;
                if (!(gx < c.ng[0] && gy < c.ng[1] && gz < c.ng[2])) continue;
                const float px = fmaf((float)gx + 0.5f, c.s_g, c.origin[0]);
                const float X = fmaf(c.R[0], px, B0), Y = fmaf(c.R[3], px, B1), Z = fmaf(c.R[6], px, B2);
                float u, v;
                int iu, iv;
                if (!project(c.Kd, PINHOLE, X, Y, Z, u, v)) continue;
                if (!nearest_pixel(u, v, c.dw, c.dh, iu, iv)) continue;
                const uint32_t D = __ldg(depth + (size_t)iv * c.dw + iu);
                if (D == 0u) continue;
                const float d = (float)D * 0.001f;
                const float sdf = d - Z;
                if (sdf < -c.mu) continue;
                if (!FREE_SPACE && sdf > c.mu) continue;
                const float t = fminf(1.0f, sdf * c.inv_mu);
                const size_t o = ((size_t)gz * c.ng[1] + gy) * c.ng[0] + gx;
                const uint32_t w = W[o];
                const float wf = (float)w;
                F[o] = __fdiv_rn(fmaf(F[o], wf, t), wf + 1.0f);
                W[o] = (uint8_t)min(w + 1u, (uint32_t)c.max_weight);
                ++count;
            }
        }
    }
    count = __reduce_add_sync(0xffffffffu, count);
    if (lane == 0 && count) atomicAdd(&ctr->geo_updated, (unsigned long long)count);
}

// ----------------------------------------------------- gate recording ----
// Adjoint gate recording: the colour voxels recorded by the band kernel that
// also pass Eq. 5, Eq. 6 (frustum, D > 0) and Eq. 7 in this frame are
// appended to the (frame, voxel) pair list: the set S_k of the photometric
// loss, which does not depend on the HD camera.
__global__ void __launch_bounds__(256) k_colour_gates(FrameConst c, const uint16_t* __restrict__ depth, Scratch scr,
                                                      AdjBuffers a, int frame) {
    const uint32_t nv = min(scr.ctr->n_vox, scr.vox_cap);
    for (uint32_t base = blockIdx.x * blockDim.x; base < nv; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool pass = false;
        uint32_t lin = 0;
        if (i < nv) {
            const uint2 r = scr.vox[i];
            const int kx = (int)(r.x & 0xFFFFu), ky = (int)(r.x >> 16), kz = (int)r.y;
            const float pwx = fmaf((float)kx + 0.5f, c.s_c, c.origin[0]);
            const float pwy = fmaf((float)ky + 0.5f, c.s_c, c.origin[1]);
            const float pwz = fmaf((float)kz + 0.5f, c.s_c, c.origin[2]);
            float X, Y, Z, u, v;
            int iu, iv;
            rigid(c.R, c.t, pwx, pwy, pwz, X, Y, Z);
            if (project(c.Kd, c.kd_pinhole, X, Y, Z, u, v) && nearest_pixel(u, v, c.dw, c.dh, iu, iv)) {
                const uint32_t D = __ldg(depth + (size_t)iv * c.dw + iu);
                if (D != 0u) {
                    float PdX, PdY, PdZ;
                    back_project(c, iu, iv, (float)D * 0.001f, PdX, PdY, PdZ);
                    const float ex = X - PdX, ey = Y - PdY, ez = Z - PdZ;
                    pass = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= c.sigma2;
                    lin = ((uint32_t)kz * (uint32_t)c.nc[1] + (uint32_t)ky) * (uint32_t)c.nc[0] + (uint32_t)kx;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        uint32_t pos = 0;
        const int lane = threadIdx.x & 31;
        if (lane == 0 && m) pos = atomicAdd(&a.counters[0], (uint32_t)__popc(m));
        pos = __shfl_sync(0xffffffffu, pos, 0) + __popc(m & ((1u << lane) - 1u));
        if (pass) {
            if (pos < a.pair_cap) {
                a.pair_vox[pos] = lin;
                a.pair_frame[pos] = (uint8_t)frame;
            } else {
                atomicOr(scr.err, ERR_PAIR_OVERFLOW);
            }
        }
    }
}

// ------------------------------------------------------ batched scans ----
// Bounded grid barrier (all blocks co-resident: cooperative launch).  The
// generation is read before arriving, the last block to arrive resets the
// count and advances the generation; the others wait for the advance for at
// most BARRIER_TIMEOUT_NS of wall time (%globaltimer) or BARRIER_SPINS polls,
// after which the wait gives up, sets the error word and the kernel returns.
constexpr unsigned long long BARRIER_TIMEOUT_NS = 1000000000ull;  // 1 s
constexpr unsigned BARRIER_SPINS = 1u << 28;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(BatchSync* s, unsigned nblocks) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &s->gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&s->count, 1u);
        if (arrived == nblocks - 1) {
            s->count = 0;
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (*vgen == g) {
                ++spins;
                if ((spins & 255u) == 0u &&
                    (global_ns() - t0 > BARRIER_TIMEOUT_NS || spins > BARRIER_SPINS || *(volatile unsigned*)&s->err)) {
                    atomicOr(&s->err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Per-block exclusive prefix over the scans of a per-scan count, each count
// rounded up to a multiple of `pad`; pre[n] is the total.
template <typename F>
__device__ __forceinline__ void scan_prefix(uint32_t* pre, int n, uint32_t pad, F count) {
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int i = 0; i < n; ++i) {
            pre[i] = acc;
            acc += (count(i) + pad - 1) / pad * pad;
        }
        pre[n] = acc;
    }
    __syncthreads();
}

__device__ __forceinline__ int find_scan(const uint32_t* pre, int n, uint32_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {  // last i with pre[i] <= item
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(COL_THREADS, 4) k_batch_step(const ScanDesc* __restrict__ descs, int n,
                                                            BatchSync* sync, int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColourSlot& S = reinterpret_cast<ColourSlot*>(smem_raw)[threadIdx.x >> 5];
    __shared__ uint32_t pre[MAX_BATCH + 1];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    const uint32_t warp = tid >> 5, nwarps = nthreads >> 5;

    // P0: counters of every scan (fold the previous frame into the totals), depth tiles
    if (tid < (uint32_t)n) {
        Counters* ctr = descs[tid].scr.ctr;
        ctr->tot_geo_updated += ctr->geo_updated;
        ctr->tot_col_updated += ctr->col_updated;
        ctr->tot_geo_bricks += ctr->n_geo;
        ctr->tot_col_bricks += ctr->n_col + ctr->n_col_light;
        ctr->tot_vis_bricks += ctr->n_vis;
        ctr->tot_cells += ctr->n_cells;
        ctr->tot_col_active += ctr->n_col_active;
        ctr->tot_geo_changed += ctr->n_geo_changed;
        ctr->frames += 1ull;
        ctr->n_geo = ctr->n_vis = ctr->n_col = ctr->n_col_light = 0;
        ctr->geo_next = ctr->col_next = 0;
        ctr->n_cells = ctr->n_vox = 0;
        ctr->n_col_active = ctr->n_geo_changed = 0;
        ctr->geo_updated = ctr->col_updated = 0ull;
    }
    if (tid == 0) sync->band_next = 0;
    if (blockIdx.x == 0 && *(volatile unsigned*)&sync->stall) return;  // test injection: never arrive
    scan_prefix(pre, n, 1, [&](int i) { return depth_strips(descs[i].c); });
    for (uint32_t item = warp; item < pre[n]; item += nwarps) {  // one warp per strip of four depth tiles
        const int s = find_scan(pre, n, item);
        depth_strip(descs[s].c, descs[s].depth, descs[s].scr.depth_tiles, nullptr, item - pre[s], lane);
    }
    if (!grid_barrier(sync, gridDim.x)) return;

    // P1: bricks (each scan's range padded to whole warps, so a warp never mixes scans)
    scan_prefix(pre, n, 32, [&](int i) { return (uint32_t)(descs[i].c.nb[0] * descs[i].c.nb[1] * descs[i].c.nb[2]); });
    for (uint32_t base = warp * 32; base < pre[n]; base += nthreads) {
        const uint32_t item = base + lane;
        const int s = find_scan(pre, n, base);
        const ScanDesc& d = descs[s];
        const uint32_t b = item - pre[s];
        const uint32_t nbt = (uint32_t)d.c.nb[0] * d.c.nb[1] * d.c.nb[2];
        bool geo, vis, inner;
        brick_flags(d.c, d.vol.summ, d.scr.depth_tiles, b, b < nbt, geo, vis, inner);
        append(geo, geo_entry(d.c, b, inner), &d.scr.ctr->n_geo, d.scr.geo_list);
        append(vis, b, &d.scr.ctr->n_vis, d.scr.vis_list);
    }
    if (!grid_barrier(sync, gridDim.x)) return;

    // P2: geometry, one warp per tile of `tile` consecutive listed bricks of a scan
    scan_prefix(pre, n, 1, [&](int i) { return (descs[i].scr.ctr->n_geo + tile - 1) / tile; });
    for (uint32_t item = warp; item < pre[n]; item += nwarps) {
        const int s = find_scan(pre, n, item);
        const ScanDesc& d = descs[s];
        const uint32_t k0 = (item - pre[s]) * tile, k1 = min(k0 + (uint32_t)tile, d.scr.ctr->n_geo);
        uint32_t count = 0, changed = 0;
        const bool aligned = d.c.ng[0] % BRICK == 0 && d.c.ng[1] % BRICK == 0 && d.c.ng[2] % BRICK == 0;
        for (uint32_t k = k0; k < k1; ++k) {
            const uint32_t e = d.scr.geo_list[k];
            const BrickAt at = geo_brick(d.c, e);
            const DepthMm dm{d.depth};
            // the usual camera and mode: without the per-voxel image tests for
            // bricks inside the image and without bounds tests for whole-brick
            // volumes; the general form handles every other brick
            if (d.c.kd_pinhole && d.c.free_space && aligned) {
                if (e & GEO_INNER)
                    geometry_brick<true, true, true, true>(d.c, d.vol, dm, at, lane, count, changed);
                else
                    geometry_brick<true, true, true, false>(d.c, d.vol, dm, at, lane, count, changed);
            } else if (d.c.kd_pinhole && d.c.free_space)
                geometry_brick<true, true>(d.c, d.vol, dm, at, lane, count, changed);
            else if (d.c.kd_pinhole)
                geometry_brick<true, false>(d.c, d.vol, dm, at, lane, count, changed);
            else if (d.c.free_space)
                geometry_brick<false, true>(d.c, d.vol, dm, at, lane, count, changed);
            else
                geometry_brick<false, false>(d.c, d.vol, dm, at, lane, count, changed);
        }
        count = __reduce_add_sync(full, count);
        if (lane == 0) {
            if (count) atomicAdd(&d.scr.ctr->geo_updated, (unsigned long long)count);
            if (changed) atomicAdd(&d.scr.ctr->n_geo_changed, changed);
        }
    }
    if (!grid_barrier(sync, gridDim.x)) return;

    // P3: colour candidates
    scan_prefix(pre, n, 32, [&](int i) { return descs[i].scr.ctr->n_vis; });
    for (uint32_t base = warp * 32; base < pre[n]; base += nthreads) {
        const uint32_t item = base + lane;
        const int s = find_scan(pre, n, base);
        const ScanDesc& d = descs[s];
        const uint32_t i = item - pre[s];
        const bool in = i < d.scr.ctr->n_vis;
        const uint32_t b = in ? d.scr.vis_list[i] : 0u;
        append(in && colour_candidate(d.c, d.vol.summ, b), b, &d.scr.ctr->n_col, d.scr.col_list);
    }
    if (!grid_barrier(sync, gridDim.x)) return;

    // P4: band gate, one warp per tile of candidates, taken with an atomic counter
    scan_prefix(pre, n, 1, [&](int i) { return (descs[i].scr.ctr->n_col + tile - 1) / tile; });
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&sync->band_next, 1u);
        item = __shfl_sync(full, item, 0);
        if (item >= pre[n]) break;
        const int s = find_scan(pre, n, item);
        const ScanDesc& d = descs[s];
        uint32_t count = 0, n_active = 0, n_cells = 0, nstage = 0;
        const uint32_t k0 = (item - pre[s]) * tile, k1 = min(k0 + (uint32_t)tile, d.scr.ctr->n_col);
        for (uint32_t k = k0; k < k1; ++k) {
            band_brick(d.c, d.vol, d.depth, d.rgb, d.scr, S, d.scr.col_list[k], lane, count, n_active, n_cells,
                       nstage);
            __syncwarp();
        }
        band_flush(d.c, d.vol, d.depth, d.rgb, d.scr, S, lane, count, nstage);  // the records are this scan's
        count = __reduce_add_sync(full, count);
        if (lane == 0) {
            if (count) atomicAdd(&d.scr.ctr->col_updated, (unsigned long long)count);
            if (n_active) atomicAdd(&d.scr.ctr->n_col_active, n_active);
            if (n_cells) atomicAdd(&d.scr.ctr->n_cells, n_cells);
        }
    }
    if (!grid_barrier(sync, gridDim.x)) return;

    // P5: colour voxels that passed the band gate
    scan_prefix(pre, n, 32, [&](int i) { return min(descs[i].scr.ctr->n_vox, descs[i].scr.vox_cap); });
    for (uint32_t base = warp * 32; base < pre[n]; base += nthreads) {
        const uint32_t item = base + lane;
        const int s = find_scan(pre, n, base);
        const ScanDesc& d = descs[s];
        const uint32_t i = item - pre[s];
        bool upd = false;
        if (i < min(d.scr.ctr->n_vox, d.scr.vox_cap)) {
            const uint2 r = d.scr.vox[i];
            upd = colour_after_band(d.c, d.vol.C, d.depth, d.rgb, (int)(r.x & 0xFFFFu), (int)(r.x >> 16), (int)r.y);
        }
        const uint32_t cnt = __popc(__ballot_sync(full, upd));
        if (lane == 0 && cnt) atomicAdd(&d.scr.ctr->col_updated, (unsigned long long)cnt);
    }
}

__global__ void k_init_summaries(BrickSummary* summ, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        BrickSummary s;
        s.fmin = __int_as_float(0x7f800000);
        s.fmax = __int_as_float(0xff800000);
        s.wmin = 0;
        s.flags = 0;
        summ[i] = s;
    }
}

}  // namespace

// --------------------------------------------------------------- launch ---
cudaError_t launch_init_summaries(BrickSummary* summ, int64_t n, cudaStream_t stream) {
    if (n > 0) k_init_summaries<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(summ, n);
    return cudaGetLastError();
}

int geometry_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_geometry<true, true, true>, GEO_THREADS, 0);
    return n > 0 ? n : 1;
}

int geometry_linear_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_geometry_linear<true, true>, GEO_THREADS, 0);
    return n > 0 ? n : 1;
}

size_t colour_smem_bytes() { return sizeof(ColourSlot) * (COL_THREADS / 32); }

int colour_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_colour_band, COL_THREADS, colour_smem_bytes());
    return n > 0 ? n : 1;
}

int fused_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<true, true>, COL_THREADS, colour_smem_bytes());
    return n > 0 ? n : 1;
}

int voxel_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_colour_voxels, 256, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_frame_pre(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                             cudaStream_t stream, cudaEvent_t* ev) {
    auto mark = [&](int i) {
        if (ev && ev[i]) cudaEventRecord(ev[i], stream);
    };
    mark(0);
    cudaError_t e = launch_chained(k_depth_tiles, depth_tiles_grid(c), dim3(TILES_THREADS), 0, stream, c, depth,
                                   s.depth_tiles, s.ctr, s.depth_m);
    mark(1);
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    if (e == cudaSuccess)
        e = launch_chained(k_bricks, dim3((nbt + BRICK_THREADS - 1) / BRICK_THREADS), dim3(BRICK_THREADS), 0, stream,
                           c, v.summ, s.depth_tiles, s.ctr, s.geo_list, s.vis_list, s.bstate, s.fsync);
    if (e == cudaSuccess && c.fused) {
        unsigned gn = (nbt + 255) / 256;
        if (gn > 1024u) gn = 1024u;
        e = launch_chained(k_need, dim3(gn), dim3(256), 0, stream, c, s);
    }
    mark(2);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_frame_post(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                              const uint8_t* rgb, const LaunchGrids& g, cudaStream_t stream, cudaEvent_t* ev,
                              cudaEvent_t list_done) {
    auto mark = [&](int i) {
        if (ev && ev[i]) cudaEventRecord(ev[i], stream);
    };
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    cudaError_t e = cudaSuccess;
    if (c.fused) {
        // geometry, colour candidates and band gate in one launch: its time
        // is the geometry phase's; the colour-list and band phases are empty
        const bool aligned = c.ng[0] % BRICK == 0 && c.ng[1] % BRICK == 0 && c.ng[2] % BRICK == 0;
        auto k = c.free_space ? (aligned ? k_fused<true, true> : k_fused<true, false>)
                              : (aligned ? k_fused<false, true> : k_fused<false, false>);
        e = launch_chained(k, dim3(g.fuse), dim3(COL_THREADS), colour_smem_bytes(), stream, c, v, depth, rgb, s);
        mark(3);
        if (list_done) cudaEventRecord(list_done, stream);
        mark(4);
        mark(5);
    } else {
        e = launch_k_geometry(c, v, s, g.geo, stream);
        mark(3);
        unsigned gl = (nbt + LIST_THREADS - 1) / LIST_THREADS;
        if (gl > 1024u) gl = 1024u;
        if (e == cudaSuccess)
            e = launch_chained(k_colour_list, dim3(gl), dim3(LIST_THREADS), 0, stream, c, v.summ, s.ctr, s.vis_list,
                               s.col_list, s.col_act);
        if (list_done) cudaEventRecord(list_done, stream);
        mark(4);
        if (e == cudaSuccess)
            e = launch_chained(k_colour_band, dim3(g.col), dim3(COL_THREADS), colour_smem_bytes(), stream, c, v, depth,
                               rgb, s);
        mark(5);
    }
    if (e == cudaSuccess)
        e = launch_chained(k_colour_voxels, dim3(g.vox), dim3(256), 0, stream, c, v, depth, rgb, s);
    mark(6);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_frame(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                         const uint8_t* rgb, const LaunchGrids& g, cudaStream_t stream, cudaEvent_t* ev) {
    cudaError_t e = launch_frame_pre(c, v, s, depth, stream, ev);
    if (e == cudaSuccess) e = launch_frame_post(c, v, s, depth, rgb, g, stream, ev, nullptr);
    return e;
}

cudaError_t launch_geometry_static(const FrameConst& c, float* F, uint8_t* W, const uint16_t* depth, Counters* ctr,
                                   uint32_t* tiles, uint32_t* geo_list, int grid_geo, cudaStream_t stream) {
    k_depth_tiles<<<depth_tiles_grid(c), TILES_THREADS, 0, stream>>>(c, depth, tiles, ctr, nullptr);
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    k_bricks_static<<<(nbt + 255) / 256, 256, 0, stream>>>(c, tiles, ctr, geo_list);
    if (c.kd_pinhole && c.free_space)
        k_geometry_linear<true, true><<<grid_geo, GEO_THREADS, 0, stream>>>(c, F, W, depth, ctr, geo_list);
    else if (c.kd_pinhole)
        k_geometry_linear<true, false><<<grid_geo, GEO_THREADS, 0, stream>>>(c, F, W, depth, ctr, geo_list);
    else if (c.free_space)
        k_geometry_linear<false, true><<<grid_geo, GEO_THREADS, 0, stream>>>(c, F, W, depth, ctr, geo_list);
    else
        k_geometry_linear<false, false><<<grid_geo, GEO_THREADS, 0, stream>>>(c, F, W, depth, ctr, geo_list);
    return cudaGetLastError();
}

cudaError_t launch_frame_record(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                                const LaunchGrids& g, const AdjBuffers& a, int frame, cudaStream_t stream) {
    k_depth_tiles<<<depth_tiles_grid(c), TILES_THREADS, 0, stream>>>(c, depth, s.depth_tiles, s.ctr, s.depth_m);
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    k_bricks<<<(nbt + BRICK_THREADS - 1) / BRICK_THREADS, BRICK_THREADS, 0, stream>>>(c, v.summ, s.depth_tiles, s.ctr,
                                                                                     s.geo_list, s.vis_list, s.bstate,
                                                                                     s.fsync);
    launch_k_geometry(c, v, s, g.geo, stream);
    unsigned gl = (nbt + LIST_THREADS - 1) / LIST_THREADS;
    if (gl > 1024u) gl = 1024u;
    k_colour_list<<<gl, LIST_THREADS, 0, stream>>>(c, v.summ, s.ctr, s.vis_list, s.col_list, s.col_act);
    k_colour_band<<<g.col, COL_THREADS, colour_smem_bytes(), stream>>>(c, v, depth, nullptr, s);
    k_colour_gates<<<g.vox, 256, 0, stream>>>(c, depth, s, a, frame);
    return cudaGetLastError();
}

size_t batch_smem_bytes() { return colour_smem_bytes(); }

int batch_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step, COL_THREADS, batch_smem_bytes());
    return n > 0 ? n : 1;
}

cudaError_t launch_batch_step(const ScanDesc* descs, int n, BatchSync* sync, int grid, int tile, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(COL_THREADS);
    cfg.dynamicSmemBytes = batch_smem_bytes();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks co-resident: the grid barrier can complete
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_step, descs, n, sync, tile);
}

}  // namespace tsdf
