// Per-frame fusion kernels: depth tiles, brick culling, geometry (TSDF)
// update, colour work list and colour update (Section IV.B).
//
// Order per frame on one stream:
//   k_depth_tiles   min / max valid depth of each 16x16 depth tile; zeroes counters
//   k_bricks        conservative per-brick visibility -> geometry and visible lists
//   k_geometry      persistent: TSDF update of each listed brick, brick summaries
//   k_colour_list   visible bricks whose 3x3x3 neighbourhood can hold |F| <= band
//   k_colour        persistent: colour update of the colour voxels each listed
//                   geometry brick owns, against a shared-memory geometry tile
// Culling only removes work whose every voxel the per-voxel logic would skip
// or leave unchanged, so results do not depend on it.
#include <cfloat>
#include <cstdint>

#include "common.cuh"

namespace tsdf {
namespace {

constexpr int GEO_THREADS = 128;  // 4 voxels per thread, one brick per block iteration
constexpr int COL_THREADS = 256;
constexpr int TILE_G = BRICK + 2;          // geometry tile edge: brick + 1-voxel halo each side
constexpr int TILE_G3 = TILE_G * TILE_G * TILE_G;
constexpr int CELLS = BRICK + 1;           // trilinear cells whose corners lie in the tile
constexpr int CELLS3 = CELLS * CELLS * CELLS;
constexpr float CELL_EPS = 1e-5f;          // bound on trilinear overshoot of the corner range

// ------------------------------------------------------------- helpers ---
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

// Nearest pixel, half-up, bounds tested in float before conversion.
__device__ __forceinline__ bool nearest_pixel(float u, float v, int W, int H, int& iu, int& iv) {
    float fu = floorf(u + 0.5f), fv = floorf(v + 0.5f);
    if (!(fu >= 0.0f && fu <= (float)(W - 1) && fv >= 0.0f && fv <= (float)(H - 1))) return false;
    iu = (int)fu;
    iv = (int)fv;
    return true;
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

// ------------------------------------------------------- depth tiles ----
__global__ void __launch_bounds__(256) k_depth_tiles(FrameConst c, const uint16_t* __restrict__ depth,
                                                     uint32_t* __restrict__ tiles, Counters* __restrict__ ctr) {
    __shared__ uint32_t s_min[8], s_max[8];
    int px = blockIdx.x * TILE_PX + threadIdx.x;
    int py = blockIdx.y * TILE_PX + threadIdx.y;
    uint32_t D = (px < c.dw && py < c.dh) ? depth[(size_t)py * c.dw + px] : 0u;
    uint32_t mn = D ? D : 0xFFFFu, mx = D;
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    int tid = threadIdx.y * TILE_PX + threadIdx.x;
    if ((tid & 31) == 0) { s_min[tid >> 5] = mn; s_max[tid >> 5] = mx; }
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < 8; ++i) { mn = min(mn, s_min[i]); mx = max(mx, s_max[i]); }
        tiles[blockIdx.y * c.tiles_x + blockIdx.x] = mn | (mx << 16);
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            // fold the previous frame's counters into the running totals
            ctr->tot_geo_updated += ctr->geo_updated;
            ctr->tot_col_updated += ctr->col_updated;
            ctr->tot_geo_bricks += ctr->n_geo;
            ctr->tot_col_bricks += ctr->n_col;
            ctr->tot_vis_bricks += ctr->n_vis;
            ctr->frames += 1ull;
            ctr->n_geo = ctr->n_vis = ctr->n_col = 0;
            ctr->geo_next = ctr->col_next = 0;
            ctr->geo_updated = ctr->col_updated = 0ull;
        }
    }
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
// (all F = 1, all w = max_weight), where (1 * w + 1) / (w + 1) = 1.
__global__ void __launch_bounds__(256) k_bricks(FrameConst c, const BrickSummary* __restrict__ summ,
                                                const uint32_t* __restrict__ tiles, Counters* __restrict__ ctr,
                                                uint32_t* __restrict__ geo_list, uint32_t* __restrict__ vis_list) {
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    bool in = b < nbt;
    bool vis = in, geo = in;
    if (in && c.culling) {
        int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        float lo[3], hi[3];
        int bc[3] = {bx, by, bz};
        for (int a = 0; a < 3; ++a) {
            lo[a] = c.origin[a] + ((float)(bc[a] * BRICK) - 0.5f) * c.s_g;
            hi[a] = c.origin[a] + ((float)(bc[a] * BRICK + BRICK) + 0.5f) * c.s_g;
        }
        float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX;
        float zmin = FLT_MAX, zmax = -FLT_MAX;
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
            zmax = fmaxf(zmax, Z);
            if (zh <= 1e-4f) { straddle = true; continue; }
            float u = xh / zh, v = yh / zh;
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
        }
        int px0 = 0, px1 = c.dw - 1, py0 = 0, py1 = c.dh - 1;
        if (!straddle) {
            // beyond the image by more than the padding: invisible
            if (umax < -2.0f || vmax < -2.0f || umin > (float)c.dw + 1.0f || vmin > (float)c.dh + 1.0f) {
                vis = false;
            } else {
                // clamp before converting so the integer bounds cannot overflow
                umin = fmaxf(umin, -4.0f); umax = fminf(umax, (float)c.dw + 4.0f);
                vmin = fmaxf(vmin, -4.0f); vmax = fminf(vmax, (float)c.dh + 4.0f);
                px0 = max(0, (int)floorf(umin) - 2); px1 = min(c.dw - 1, (int)ceilf(umax) + 2);
                py0 = max(0, (int)floorf(vmin) - 2); py1 = min(c.dh - 1, (int)ceilf(vmax) + 2);
            }
        }
        uint32_t dmin = 0xFFFFu, dmax = 0u;
        if (vis) {
            int tx0 = px0 / TILE_PX, tx1 = px1 / TILE_PX, ty0 = py0 / TILE_PX, ty1 = py1 / TILE_PX;
            if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 64) {
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx) {
                        uint32_t tv = tiles[ty * c.tiles_x + tx];
                        dmin = min(dmin, tv & 0xFFFFu);
                        dmax = max(dmax, tv >> 16);
                    }
            } else {
                dmin = 1u;
                dmax = 0xFFFFu;
            }
            if (dmax == 0u) vis = false;                                   // no measurement under it
            else if (zmin > (float)dmax * 0.001f + c.cull_behind) vis = false;  // hidden behind every surface
        }
        geo = vis;
        if (vis) {
            const BrickSummary s = summ[b];
            bool sat = c.free_space == 0 || (s.fmin == 1.0f && s.wmin == (uint32_t)c.max_weight);
            if (sat && zmax < (float)dmin * 0.001f - c.mu - 2e-3f) geo = false;
        }
    }
    append(geo, b, &ctr->n_geo, geo_list);
    append(vis, b, &ctr->n_vis, vis_list);
}

// ---------------------------------------------------------- geometry ----
// TSDF update (the KinectFusion step the paper inherits, Section III):
//   D = depth at the nearest pixel of the voxel centre (Eq. 6); D = 0 skipped
//   sdf = D * 0.001 - Z; sdf < -mu skipped; (free space off: sdf > mu skipped)
//   t = min(1, sdf * (1/mu)); F <- fmaf(F, w, t) / (w + 1); w <- min(w+1, max_w)
// Thread t of a block owns voxels 4t..4t+3 of the brick (same y and z), so the
// y/z part of Eq. 5 is computed once per thread; F and w move as one float4
// and one 32-bit word, a warp covering 512 + 128 contiguous bytes.
__global__ void __launch_bounds__(GEO_THREADS) k_geometry(FrameConst c, Volumes vol, const uint16_t* __restrict__ depth,
                                                          Counters* __restrict__ ctr,
                                                          const uint32_t* __restrict__ list) {
    __shared__ uint32_t s_item;
    __shared__ float s_fmin[GEO_THREADS / 32], s_fmax[GEO_THREADS / 32];
    __shared__ uint32_t s_wmin[GEO_THREADS / 32];
    const int tid = threadIdx.x;
    const int lx = (tid & 1) * 4, ly = (tid >> 1) & 7, lz = tid >> 4;
    const uint32_t n = ctr->n_geo;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&ctr->geo_next, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n) break;
        const uint32_t b = list[item];
        const int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
        const int gx0 = bx * BRICK + lx, gy = by * BRICK + ly, gz = bz * BRICK + lz;
        const float py = fmaf((float)gy + 0.5f, c.s_g, c.origin[1]);
        const float pz = fmaf((float)gz + 0.5f, c.s_g, c.origin[2]);
        const float B0 = fmaf(c.R[1], py, fmaf(c.R[2], pz, c.t[0]));
        const float B1 = fmaf(c.R[4], py, fmaf(c.R[5], pz, c.t[1]));
        const float B2 = fmaf(c.R[7], py, fmaf(c.R[8], pz, c.t[2]));
        const bool yz_in = gy < c.ng[1] && gz < c.ng[2];
        float tv[4];
        uint32_t upd = 0, inb = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            tv[j] = 0.0f;
            const int gx = gx0 + j;
            if (!(yz_in && gx < c.ng[0])) continue;
            inb |= 1u << j;
            const float px = fmaf((float)gx + 0.5f, c.s_g, c.origin[0]);
            const float X = fmaf(c.R[0], px, B0), Y = fmaf(c.R[3], px, B1), Z = fmaf(c.R[6], px, B2);
            float u, v;
            int iu, iv;
            if (!project(c.Kd, c.kd_pinhole, X, Y, Z, u, v)) continue;
            if (!nearest_pixel(u, v, c.dw, c.dh, iu, iv)) continue;
            const uint32_t D = __ldg(depth + (size_t)iv * c.dw + iu);
            if (D == 0u) continue;
            const float d = (float)D * 0.001f;
            const float sdf = d - Z;
            if (sdf < -c.mu) continue;
            if (!c.free_space && sdf > c.mu) continue;
            tv[j] = fminf(1.0f, sdf * c.inv_mu);
            upd |= 1u << j;
        }
        if (__syncthreads_or(upd != 0u)) {
            const size_t base = (size_t)b * BRICK_VOX + (size_t)tid * 4;
            float4 f = *reinterpret_cast<const float4*>(vol.F + base);
            uint32_t wv = *reinterpret_cast<const uint32_t*>(vol.W + base);
            float fv[4] = {f.x, f.y, f.z, f.w};
            uint32_t wn = wv;
            float fmn = FLT_MAX, fmx = -FLT_MAX;
            uint32_t wmn = 0xFFFFFFFFu;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t w = (wv >> (8 * j)) & 0xFFu;
                if (upd & (1u << j)) {
                    const float wf = (float)w;
                    fv[j] = __fdiv_rn(fmaf(fv[j], wf, tv[j]), wf + 1.0f);
                    w = min(w + 1u, (uint32_t)c.max_weight);
                    wn = (wn & ~(0xFFu << (8 * j))) | (w << (8 * j));
                }
                if (inb & (1u << j)) {
                    wmn = min(wmn, w);
                    if (w) { fmn = fminf(fmn, fv[j]); fmx = fmaxf(fmx, fv[j]); }
                }
            }
            if (upd) {
                *reinterpret_cast<float4*>(vol.F + base) = make_float4(fv[0], fv[1], fv[2], fv[3]);
                *reinterpret_cast<uint32_t*>(vol.W + base) = wn;
            }
            // brick summary: block reduction of min/max
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                fmn = fminf(fmn, __shfl_xor_sync(0xffffffffu, fmn, o));
                fmx = fmaxf(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
            }
            wmn = __reduce_min_sync(0xffffffffu, wmn);
            const uint32_t cnt = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(upd));
            if ((tid & 31) == 0) {
                s_fmin[tid >> 5] = fmn;
                s_fmax[tid >> 5] = fmx;
                s_wmin[tid >> 5] = wmn;
                if (cnt) atomicAdd(&ctr->geo_updated, (unsigned long long)cnt);
            }
            __syncthreads();
            if (tid == 0) {
                for (int i = 1; i < GEO_THREADS / 32; ++i) {
                    fmn = fminf(fmn, s_fmin[i]);
                    fmx = fmaxf(fmx, s_fmax[i]);
                    wmn = min(wmn, s_wmin[i]);
                }
                BrickSummary s;
                s.fmin = fmn == FLT_MAX ? __int_as_float(0x7f800000) : fmn;
                s.fmax = fmx == -FLT_MAX ? __int_as_float(0xff800000) : fmx;
                s.wmin = wmn == 0xFFFFFFFFu ? 0u : wmn;
                s.pad = 0;
                vol.summ[b] = s;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- colour list ----
// A visible geometry brick goes to the colour list when the F range of its
// 3x3x3 brick neighbourhood (observed voxels only) meets [-band, band]: the
// trilinear TSDF of any colour voxel it owns is a convex combination of
// corner values from that neighbourhood, up to CELL_EPS of rounding.
__global__ void __launch_bounds__(256) k_colour_list(FrameConst c, const BrickSummary* __restrict__ summ,
                                                     Counters* __restrict__ ctr, const uint32_t* __restrict__ vis_list,
                                                     uint32_t* __restrict__ col_list) {
    const uint32_t n = ctr->n_vis;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool act = false;
        uint32_t b = 0;
        if (i < n) {
            b = vis_list[i];
            act = true;
            if (c.culling) {
                const int bx = b % c.nb[0], by = (b / c.nb[0]) % c.nb[1], bz = b / (c.nb[0] * c.nb[1]);
                float mn = FLT_MAX, mx = -FLT_MAX;
                for (int dz = -1; dz <= 1; ++dz) {
                    const int z = bz + dz;
                    if (z < 0 || z >= c.nb[2]) continue;
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int y = by + dy;
                        if (y < 0 || y >= c.nb[1]) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int x = bx + dx;
                            if (x < 0 || x >= c.nb[0]) continue;
                            const BrickSummary s = summ[((size_t)z * c.nb[1] + y) * c.nb[0] + x];
                            mn = fminf(mn, s.fmin);
                            mx = fmaxf(mx, s.fmax);
                        }
                    }
                }
                act = mn <= c.band + CELL_EPS && mx >= -c.band - CELL_EPS;
            }
        }
        append(act, b, &ctr->n_col, col_list);
    }
}

// ------------------------------------------------------------ colour ----
// Range of colour indices whose centres lie in geometry brick bb along one
// axis: 16 bb Nc <= (2k + 1) Ng < 16 (bb + 1) Nc (exact integer arithmetic, so
// every colour voxel belongs to exactly one geometry brick).
__device__ __forceinline__ void owned_range(int bb, int ng, int nc, int& k0, int& k1) {
    auto lo = [&](long long B) -> long long {  // smallest k with (2k+1) ng >= 16 B nc
        long long num = 16ll * B * nc - ng;  // 2k ng >= num
        if (num <= 0) return 0;
        long long den = 2ll * ng;
        return (num + den - 1) / den;
    };
    k0 = (int)min((long long)nc, lo(bb));
    k1 = (int)min((long long)nc, lo(bb + 1));  // exclusive
}

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

// Colour update (Section IV.B) of the colour voxels a geometry brick owns.
// The block stages the brick's geometry plus a one-voxel halo (10^3 F and w,
// post-update) in shared memory, marks which of the 9^3 trilinear cells can
// pass the band gate (all 8 corners observed and the corner range meets
// [-band, band]), and then runs, per colour voxel whose cell is marked:
//   Eq. 5 -> Eq. 6 -> D > 0 -> Eq. 7 sigma gate -> trilinear band gate
//   -> Eq. 3-4 -> HD sample -> Eq. 9 (integer, half-up) or Eq. 8-10.
// The cell test is conservative, so the gates decide exactly as written.
__global__ void __launch_bounds__(COL_THREADS) k_colour(FrameConst c, Volumes vol, const uint16_t* __restrict__ depth,
                                                        const uint8_t* __restrict__ rgb, Counters* __restrict__ ctr,
                                                        const uint32_t* __restrict__ list, uint32_t* __restrict__ err) {
    __shared__ float sF[TILE_G3];
    __shared__ uint8_t sW[TILE_G3];
    __shared__ uint8_t sCell[CELLS3];
    __shared__ uint32_t s_item;
    const int tid = threadIdx.x;
    const uint32_t n = ctr->n_col;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&ctr->col_next, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n) break;
        const uint32_t b = list[item];
        const int bb[3] = {(int)(b % c.nb[0]), (int)((b / c.nb[0]) % c.nb[1]), (int)(b / (c.nb[0] * c.nb[1]))};
        const int t0[3] = {bb[0] * BRICK - 1, bb[1] * BRICK - 1, bb[2] * BRICK - 1};
        for (int i = tid; i < TILE_G3; i += COL_THREADS) {
            const int x = t0[0] + i % TILE_G, y = t0[1] + (i / TILE_G) % TILE_G, z = t0[2] + i / (TILE_G * TILE_G);
            float f = 0.0f;
            uint8_t w = 0;
            if (x >= 0 && y >= 0 && z >= 0 && x < c.ng[0] && y < c.ng[1] && z < c.ng[2]) {
                const int64_t o = brick_offset(x, y, z, c.nb);
                f = vol.F[o];
                w = vol.W[o];
            }
            sF[i] = f;
            sW[i] = w;
        }
        __syncthreads();
        for (int i = tid; i < CELLS3; i += COL_THREADS) {
            const int x = i % CELLS, y = (i / CELLS) % CELLS, z = i / (CELLS * CELLS);
            const int o = (z * TILE_G + y) * TILE_G + x;
            bool allw = true;
            float mn = FLT_MAX, mx = -FLT_MAX;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int oo = o + (k & 1) + ((k >> 1) & 1) * TILE_G + (k >> 2) * TILE_G * TILE_G;
                allw = allw && sW[oo] != 0;
                mn = fminf(mn, sF[oo]);
                mx = fmaxf(mx, sF[oo]);
            }
            bool act = allw;
            if (c.culling) act = act && mn <= c.band + CELL_EPS && mx >= -c.band - CELL_EPS;
            sCell[i] = act ? 1 : 0;
        }
        __syncthreads();
        int k0[3], k1[3];
        for (int a = 0; a < 3; ++a) owned_range(bb[a], c.ng[a], c.nc[a], k0[a], k1[a]);
        const int ex = k1[0] - k0[0], ey = k1[1] - k0[1], ez = k1[2] - k0[2];
        const int nvox = ex * ey * ez;
        uint32_t cnt = 0;
        for (int i = tid; i < nvox; i += COL_THREADS) {
            const int kx = k0[0] + i % ex, ky = k0[1] + (i / ex) % ey, kz = k0[2] + i / (ex * ey);
            const float pw[3] = {fmaf((float)kx + 0.5f, c.s_c, c.origin[0]), fmaf((float)ky + 0.5f, c.s_c, c.origin[1]),
                                 fmaf((float)kz + 0.5f, c.s_c, c.origin[2])};
            float g[3], i0[3];
            int cell[3];
            bool range_ok = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                g[a] = fmaf(pw[a] - c.origin[a], c.inv_sg, -0.5f);
                i0[a] = floorf(g[a]);
                cell[a] = (int)i0[a] - t0[a];
                range_ok = range_ok && cell[a] >= 0 && cell[a] < CELLS;
            }
            if (!range_ok) {
                atomicOr(err, ERR_TILE_RANGE);
                continue;
            }
            if (!sCell[(cell[2] * CELLS + cell[1]) * CELLS + cell[0]]) continue;
            float X, Y, Z;
            rigid(c.R, c.t, pw[0], pw[1], pw[2], X, Y, Z);
            float u, v;
            int iu, iv;
            if (!project(c.Kd, c.kd_pinhole, X, Y, Z, u, v)) continue;
            if (!nearest_pixel(u, v, c.dw, c.dh, iu, iv)) continue;
            const uint32_t D = __ldg(depth + (size_t)iv * c.dw + iu);
            if (D == 0u) continue;
            const float d = (float)D * 0.001f;
            float PdX, PdY, PdZ;
            back_project(c, iu, iv, d, PdX, PdY, PdZ);
            const float ex_ = X - PdX, ey_ = Y - PdY, ez_ = Z - PdZ;
            const float dist2 = fmaf(ex_, ex_, fmaf(ey_, ey_, ez_ * ez_));
            if (dist2 > c.sigma2) continue;
            // trilinear TSDF: lerp along x, then y, then z
            const int o = (cell[2] * TILE_G + cell[1]) * TILE_G + cell[0];
            const float fx = g[0] - i0[0], fy = g[1] - i0[1], fz = g[2] - i0[2];
            const float c00 = lerp(sF[o], sF[o + 1], fx);
            const float c10 = lerp(sF[o + TILE_G], sF[o + TILE_G + 1], fx);
            const float c01 = lerp(sF[o + TILE_G * TILE_G], sF[o + TILE_G * TILE_G + 1], fx);
            const float c11 = lerp(sF[o + TILE_G * TILE_G + TILE_G], sF[o + TILE_G * TILE_G + TILE_G + 1], fx);
            const float c0 = lerp(c00, c10, fy);
            const float c1 = lerp(c01, c11, fy);
            const float Ft = lerp(c0, c1, fz);
            if (!(fabsf(Ft) <= c.band)) continue;
            float Xh, Yh, Zh;
            rigid(c.Rc, c.tc, X, Y, Z, Xh, Yh, Zh);
            float uh, vh;
            if (!project(c.Kr, c.kr_pinhole, Xh, Yh, Zh, uh, vh)) continue;
            uint32_t s[3];
            if (!sample_rgb(c, rgb, uh, vh, s)) continue;
            const int64_t co = brick_offset(kx, ky, kz, c.ncb);
            uint32_t vox = vol.C[co];
            if (c.colour_mode == 1) {
                if (!paper_normal_update(c, depth, iu, iv, PdX, PdY, PdZ, X, Y, Z, vox, s)) continue;
            } else {
                const uint32_t w = vox >> 24;
                uint32_t out = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const uint32_t cc = (vox >> (8 * k)) & 0xFFu;
                    out |= ((cc * w + s[k] + ((w + 1u) >> 1)) / (w + 1u)) << (8 * k);
                }
                const uint32_t wn = min(w + 1u, (uint32_t)c.max_weight);
                vox = out | (wn << 24);
            }
            vol.C[co] = vox;
            ++cnt;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if ((tid & 31) == 0 && cnt) atomicAdd(&ctr->col_updated, (unsigned long long)cnt);
        __syncthreads();
    }
}

__global__ void k_init_summaries(BrickSummary* summ, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        BrickSummary s;
        s.fmin = __int_as_float(0x7f800000);
        s.fmax = __int_as_float(0xff800000);
        s.wmin = 0;
        s.pad = 0;
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_geometry, GEO_THREADS, 0);
    return n > 0 ? n : 1;
}

int colour_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_colour, COL_THREADS, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_frame(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                         const uint8_t* rgb, int grid_geo, int grid_col, cudaStream_t stream, cudaEvent_t* ev) {
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], stream);
    };
    mark(0);
    dim3 tg(c.tiles_x, c.tiles_y);
    k_depth_tiles<<<tg, dim3(TILE_PX, TILE_PX), 0, stream>>>(c, depth, s.depth_tiles, s.ctr);
    mark(1);
    const uint32_t nbt = (uint32_t)c.nb[0] * c.nb[1] * c.nb[2];
    k_bricks<<<(nbt + 255) / 256, 256, 0, stream>>>(c, v.summ, s.depth_tiles, s.ctr, s.geo_list, s.vis_list);
    mark(2);
    k_geometry<<<grid_geo, GEO_THREADS, 0, stream>>>(c, v, depth, s.ctr, s.geo_list);
    mark(3);
    unsigned gl = (nbt + 255) / 256;
    if (gl > 1024u) gl = 1024u;
    k_colour_list<<<gl, 256, 0, stream>>>(c, v.summ, s.ctr, s.vis_list, s.col_list);
    mark(4);
    k_colour<<<grid_col, COL_THREADS, 0, stream>>>(c, v, depth, rgb, s.ctr, s.col_list, s.err);
    mark(5);
    return cudaGetLastError();
}

}  // namespace tsdf
