// Host side of the C ABI declared in include/tsdf.h.
//
// Frame constants are computed here in binary64 and rounded once to binary32
// (host code is compiled with -ffp-contract=off, so each product and sum is
// rounded as written):
//   R_n = R_wd^T (an exact transpose of the given floats)
//   t_n[i] = -((R[0][i] t[0] + R[1][i] t[1]) + R[2][i] t[2])   (Eq. 5 motion)
//   K_c^-1 = adjugate / det, det expanded along the first row  (Eq. 7)
//   1/mu, 1/s_g as binary32 quotients, sigma^2 as a binary32 product.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tsdf.h"
#include "api_internal.h"
#include "common.cuh"

using namespace tsdf;

namespace tsdf_host {

constexpr int64_t MAX_DIM = 4096;
constexpr int32_t MAX_IMAGE = 16384;

tsdf_status fail(tsdf_volume* v, tsdf_status s, const std::string& msg) {
    if (v) v->last_error = msg;
    return s;
}

tsdf_status cuda_fail(tsdf_volume* v, cudaError_t e, const char* where) {
    return fail(v, TSDF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(tsdf_volume* v, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (v->alloc.alloc) {
        p = v->alloc.alloc(bytes, (void*)v->stream, v->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        v->blocks.push_back({p, bytes});
        v->device_bytes += (int64_t)bytes;
    }
    return p;
}

void dev_free(tsdf_volume* v, void* p) {
    if (!p) return;
    for (size_t i = 0; i < v->blocks.size(); ++i) {
        if (v->blocks[i].p == p) {
            size_t bytes = v->blocks[i].bytes;
            if (v->alloc.free)
                v->alloc.free(p, bytes, (void*)v->stream, v->alloc.ctx);
            else
                cudaFree(p);
            v->device_bytes -= (int64_t)bytes;
            v->blocks.erase(v->blocks.begin() + (ptrdiff_t)i);
            return;
        }
    }
}

// Band-gate voxel record capacity for a volume of nbt geometry bricks.
int64_t vox_capacity(int64_t nbt) {
    return std::min<int64_t>(std::max<int64_t>(int64_t(1) << 22, nbt * 64), int64_t(1) << 28);
}

bool finite_all(const float* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Translation within MAX_COORD metres.
bool translation_ok(const float T[16]) {
    for (int i = 0; i < 3; ++i)
        if (!(std::fabs(T[i * 4 + 3]) <= MAX_COORD)) return false;
    return true;
}

// Rigid transform check: finite, bottom row (0, 0, 0, 1), |R^T R - I| <= 1e-4.
bool rigid_ok(const float T[16]) {
    if (!finite_all(T, 16)) return false;
    if (T[12] != 0.0f || T[13] != 0.0f || T[14] != 0.0f || T[15] != 1.0f) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += (double)T[k * 4 + i] * (double)T[k * 4 + j];
            if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-4) return false;
        }
    return true;
}

bool pinhole(const float K[9]) {
    return K[1] == 0.0f && K[3] == 0.0f && K[6] == 0.0f && K[7] == 0.0f && K[8] == 1.0f;
}

// K^-1 by the adjugate over the first-row determinant, binary64, rounded once.
bool invert3(const float K[9], float out[9]) {
    const double a = K[0], b = K[1], c = K[2], d = K[3], e = K[4], f = K[5], g = K[6], h = K[7], i = K[8];
    const double A = e * i - f * h;
    const double B = f * g - d * i;
    const double C = d * h - e * g;
    const double det = (a * A + b * B) + c * C;
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    const double adj[9] = {A, c * h - b * i, b * f - c * e, B, a * i - c * g, c * d - a * f, C, b * g - a * h, a * e - b * d};
    for (int k = 0; k < 9; ++k) out[k] = (float)(adj[k] / det);
    return finite_all(out, 9);
}

void frame_constants(const tsdf_volume* v, const float Kd[9], const float Kr[9], const float Twd[16],
                     const float Tdr[16], int dw, int dh, int cw, int ch, FrameConst& c) {
    std::memset(&c, 0, sizeof c);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) c.R[r * 3 + k] = Twd[k * 4 + r];
    for (int i = 0; i < 3; ++i) {
        double s = (double)Twd[0 * 4 + i] * (double)Twd[0 * 4 + 3];
        s = s + (double)Twd[1 * 4 + i] * (double)Twd[1 * 4 + 3];
        s = s + (double)Twd[2 * 4 + i] * (double)Twd[2 * 4 + 3];
        c.t[i] = (float)(-s);
    }
    std::memcpy(c.Kd, Kd, sizeof c.Kd);
    invert3(Kd, c.Kdi);
    std::memcpy(c.Kr, Kr, sizeof c.Kr);
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.Rc[r * 3 + k] = Tdr[r * 4 + k];
        c.tc[r] = Tdr[r * 4 + 3];
    }
    for (int a = 0; a < 3; ++a) {
        c.origin[a] = v->origin[a];
        c.ng[a] = v->ng[a];
        c.nc[a] = v->nc[a];
        c.nb[a] = v->nb[a];
        c.ncb[a] = v->ncb[a];
    }
    c.zoff_g = v->zoff_g;
    c.zoff_c = v->zoff_c;
    c.s_g = v->s_g;
    c.s_c = v->s_c;
    c.inv_sg = 1.0f / v->s_g;
    c.mu = v->mu;
    c.inv_mu = 1.0f / v->mu;
    c.sigma2 = v->sigma * v->sigma;
    c.band = v->band;
    c.dw = dw;
    c.dh = dh;
    c.pix_bias = 0x4B000000u * (uint32_t)(dw + 1);
    c.cw = cw;
    c.ch = ch;
    c.tiles_x = (dw + TILE_PX - 1) / TILE_PX;
    c.tiles_y = (dh + TILE_PX - 1) / TILE_PX;
    c.kd_pinhole = pinhole(Kd);
    c.kr_pinhole = pinhole(Kr);
    c.kdi_pinhole = c.Kdi[1] == 0.0f && c.Kdi[3] == 0.0f && c.Kdi[6] == 0.0f && c.Kdi[7] == 0.0f && c.Kdi[8] == 1.0f;
    c.max_weight = v->max_weight;
    c.free_space = v->free_space;
    c.sample_mode = v->sample_mode;
    c.colour_mode = v->colour_mode;
    c.culling = v->culling;
    // Beyond the farthest depth by more than max(mu, sigma) nothing can pass
    // the sdf >= -mu test nor (pinhole K_c: the back-projected point has
    // Z = d) the sigma gate; 2 mm covers binary32 rounding many times over.
    c.cull_behind = c.kdi_pinhole ? std::fmax(v->mu, v->sigma) + 2e-3f : INFINITY;
}

tsdf_status check_device_error(tsdf_volume* v) {
    uint32_t e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, v->scr.err, sizeof e, cudaMemcpyDeviceToHost, v->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(v->stream);
    if (ce != cudaSuccess) return cuda_fail(v, ce, "device status read");
    if (e) {
        cudaMemsetAsync(v->scr.err, 0, sizeof(uint32_t), v->stream);
        if (e == ERR_WAIT_TIMEOUT)
            return fail(v, TSDF_ERR_TIMEOUT, "fused frame: a bounded wait for ready colour work gave up");
        return fail(v, TSDF_ERR_DEVICE_FAULT, "device status word 0x" + std::to_string(e));
    }
    return TSDF_OK;
}

template <typename T>
tsdf_status read_volume(tsdf_volume* v, const T* brick, T* dst, const int32_t dims[3],
                        cudaError_t (*conv)(const T*, T*, const int32_t*, int, int, cudaStream_t)) {
    if (!dst) return TSDF_OK;
    if (is_device_ptr(dst)) {
        cudaError_t e = conv(brick, dst, dims, 0, dims[2], v->stream);
        return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "read-out");
    }
    const size_t slab = (size_t)dims[0] * dims[1] * BRICK;
    T* tmp = (T*)dev_alloc(v, slab * sizeof(T));
    if (!tmp) return fail(v, TSDF_ERR_OOM, "read-out staging buffer");
    tsdf_status st = TSDF_OK;
    for (int z0 = 0; z0 < dims[2] && st == TSDF_OK; z0 += BRICK) {
        const int z1 = std::min(dims[2], z0 + BRICK);
        cudaError_t e = conv(brick, tmp, dims, z0, z1, v->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + (size_t)dims[0] * dims[1] * z0, tmp, (size_t)dims[0] * dims[1] * (z1 - z0) * sizeof(T),
                                cudaMemcpyDeviceToHost, v->stream);
        if (e != cudaSuccess) st = cuda_fail(v, e, "read-out");
    }
    cudaStreamSynchronize(v->stream);
    dev_free(v, tmp);
    return st;
}

template <typename T>
tsdf_status write_volume(tsdf_volume* v, T* brick, const T* src, const int32_t dims[3],
                         cudaError_t (*conv)(T*, const T*, const int32_t*, int, int, cudaStream_t)) {
    if (!src) return TSDF_OK;
    if (is_device_ptr(src)) {
        cudaError_t e = conv(brick, src, dims, 0, dims[2], v->stream);
        return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "restore");
    }
    const size_t slab = (size_t)dims[0] * dims[1] * BRICK;
    T* tmp = (T*)dev_alloc(v, slab * sizeof(T));
    if (!tmp) return fail(v, TSDF_ERR_OOM, "restore staging buffer");
    tsdf_status st = TSDF_OK;
    for (int z0 = 0; z0 < dims[2] && st == TSDF_OK; z0 += BRICK) {
        const int z1 = std::min(dims[2], z0 + BRICK);
        cudaError_t e = cudaMemcpyAsync(tmp, src + (size_t)dims[0] * dims[1] * z0,
                                        (size_t)dims[0] * dims[1] * (z1 - z0) * sizeof(T), cudaMemcpyHostToDevice, v->stream);
        if (e == cudaSuccess) e = conv(brick, tmp, dims, z0, z1, v->stream);
        if (e != cudaSuccess) st = cuda_fail(v, e, "restore");
    }
    cudaStreamSynchronize(v->stream);
    dev_free(v, tmp);
    return st;
}

tsdf_status stage_depth(tsdf_volume* v, const uint16_t* depth_mm, tsdf_image_size dsz, int tiles,
                        const uint16_t** d_depth) {
    v->chain_ok = false;  // the caller runs a frame outside the integrate pipeline
    const size_t dbytes = (size_t)dsz.width * dsz.height * sizeof(uint16_t);
    *d_depth = depth_mm;
    if (!is_device_ptr(depth_mm)) {
        if (v->d_depth_cap < dbytes) {
            dev_free(v, v->d_depth);
            v->d_depth = (uint16_t*)dev_alloc(v, dbytes);
            v->d_depth_cap = v->d_depth ? dbytes : 0;
            if (!v->d_depth) return fail(v, TSDF_ERR_OOM, "depth staging buffer");
        }
        cudaError_t e = cudaMemcpyAsync(v->d_depth, depth_mm, dbytes, cudaMemcpyHostToDevice, v->stream);
        if (e != cudaSuccess) return cuda_fail(v, e, "depth upload");
        *d_depth = v->d_depth;
    }
    return depth_scratch(v, (size_t)tiles, dsz);
}

tsdf_status depth_scratch(tsdf_volume* v, size_t tiles, tsdf_image_size dsz) {
    const size_t tbytes = (tiles * sizeof(uint32_t) + 15) & ~(size_t)15;
    const size_t bytes = tbytes + (size_t)dsz.width * dsz.height * sizeof(float);
    if (v->depth_tiles_cap < bytes) {
        dev_free(v, v->depth_tiles);
        v->depth_tiles = (uint32_t*)dev_alloc(v, bytes);
        v->depth_tiles_cap = v->depth_tiles ? bytes : 0;
        if (!v->depth_tiles) return fail(v, TSDF_ERR_OOM, "depth tile buffer");
    }
    v->scr.depth_tiles = v->depth_tiles;
    v->scr.depth_m = reinterpret_cast<float*>(reinterpret_cast<char*>(v->depth_tiles) + tbytes);
    return TSDF_OK;
}

}  // namespace tsdf_host

using namespace tsdf_host;


namespace tsdf {
// Frame constants for the allocation-free geometry entry point: a volume
// description filled into a temporary handle and passed to the same
// frame_constants() as tsdf_integrate (geometry fields only; the colour
// fields are unused on that path).
void geometry_frame_constants(const VolumeDesc& d, const float Kd[9], const float Twd[16], int dw, int dh,
                              FrameConst& c) {
    tsdf_volume v{};
    for (int a = 0; a < 3; ++a) {
        v.ng[a] = d.ng[a];
        v.nc[a] = d.ng[a];
        v.nb[a] = (d.ng[a] + BRICK - 1) / BRICK;
        v.ncb[a] = v.nb[a];
        v.origin[a] = d.origin[a];
    }
    v.s_g = d.s_g;
    v.s_c = d.s_g;
    v.mu = d.mu;
    v.sigma = d.mu;  // the cull margin then reduces to mu, the geometry bound
    v.band = 0.0f;
    v.max_weight = d.max_weight;
    v.colour_mode = 0;
    v.sample_mode = 0;
    v.culling = 1;
    v.free_space = 1;
    const float I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    frame_constants(&v, Kd, Kd, Twd, I, dw, dh, dw, dh, c);
}
}  // namespace tsdf

// =================================================================== API ==
extern "C" {

void tsdf_params_default(tsdf_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->origin[0] = p->origin[1] = p->origin[2] = NAN;
    p->sigma = 0.020f;
    p->band = NAN;
    p->colour_mode = TSDF_COLOUR_COUNT;
    p->sample_mode = TSDF_SAMPLE_NEAREST;
    p->culling = 1;
    p->update_free_space = 1;
    p->stream = nullptr;
}

const char* tsdf_status_string(tsdf_status s) {
    switch (s) {
        case TSDF_OK: return "ok";
        case TSDF_ERR_INVALID_ARG: return "invalid argument";
        case TSDF_ERR_OOM: return "out of device memory";
        case TSDF_ERR_CUDA: return "CUDA error";
        case TSDF_ERR_TIMEOUT: return "device-side wait timed out";
        case TSDF_ERR_DEVICE_FAULT: return "device-side error recorded";
        case TSDF_ERR_IO: return "checkpoint I/O error";
    }
    return "unknown status";
}

const char* tsdf_last_error(const tsdf_volume* v) { return v ? v->last_error.c_str() : ""; }

// Per-axis colour tables (see AxisTables): the trilinear cell and fraction of
// each colour index, computed with the same binary32 operations as the band
// kernel (centre p = fmaf(k + 1/2, s_c, origin), g = fmaf(p - origin, 1/s_g,
// -1/2), i0 = floor(g), fraction g - i0); a brick owns the colour indices
// whose cell's lower corner i0 lies in it (i0 is non-decreasing in k, so the
// owned indices are a contiguous range), and the per-cell spans.
static tsdf_status build_axis_tables(tsdf_volume* v) {
    const float inv_sg = 1.0f / v->s_g;
    for (int a = 0; a < 3; ++a) {
        const int nc = v->nc[a], nb = v->nb[a];
        // on a z-slab handle the z indices are offset by the slab's global
        // index of held voxel 0 (colour zc, geometry zg)
        const long long zg = a == 2 ? v->zoff_g : 0, zc = a == 2 ? v->zoff_c : 0;
        std::vector<float> frac(nc);
        std::vector<int8_t> cell(nc);
        std::vector<long long> low(nc);  // held geometry index of each colour index's lower cell corner
        for (int k = 0; k < nc; ++k) {
            const float p = std::fmaf((float)(k + zc) + 0.5f, v->s_c, v->origin[a]);
            const float g = std::fmaf(p - v->origin[a], inv_sg, -0.5f);
            const float i0 = std::floor(g);
            frac[k] = g - i0;
            low[k] = (long long)i0 - zg;
            if (k > 0 && low[k] < low[k - 1])
                return fail(v, TSDF_ERR_INVALID_ARG, "colour grid does not fit the bricks");
        }
        std::vector<int32_t> k0(nb + 1);
        for (int bb = 0, k = 0; bb <= nb; ++bb) {  // first index whose lower corner is in brick bb or later
            while (k < nc && low[k] < 8ll * bb) ++k;
            k0[bb] = k;
        }
        std::vector<uint16_t> span((size_t)nb * BRICK, 0);
        for (int bb = 0; bb < nb; ++bb) {
            for (int k = k0[bb]; k < k0[bb + 1]; ++k) {
                const int rel = (int)(low[k] - 8ll * bb);  // 0..7 by the ownership above
                cell[k] = (int8_t)rel;
                const int j = k - k0[bb];
                if (j > 255) return fail(v, TSDF_ERR_INVALID_ARG, "colour grid does not fit the bricks");
                uint16_t& sp = span[(size_t)bb * BRICK + rel];
                if ((sp >> 8) == 0) sp = (uint16_t)(j | ((j + 1) << 8));
                else sp = (uint16_t)((sp & 0xFFu) | ((j + 1) << 8));
            }
        }
        std::vector<uint16_t> info(nb, 0);
        for (int bb = 0; bb < nb; ++bb) {
            uint32_t mask = 0, most = 0;
            for (int cl = 0; cl < BRICK; ++cl) {
                const uint16_t sp = span[(size_t)bb * BRICK + cl];
                const uint32_t n = (sp >> 8) - (sp & 0xFFu);
                if (sp >> 8) mask |= 1u << cl;
                most = std::max(most, (sp >> 8) ? n : 0u);
            }
            info[bb] = (uint16_t)(mask | (most << 9));
        }
        uint16_t* d_info = (uint16_t*)dev_alloc(v, nb * sizeof(uint16_t));
        float* d_frac = (float*)dev_alloc(v, nc * sizeof(float));
        int8_t* d_cell = (int8_t*)dev_alloc(v, nc);
        int32_t* d_k0 = (int32_t*)dev_alloc(v, (nb + 1) * sizeof(int32_t));
        uint16_t* d_span = (uint16_t*)dev_alloc(v, (size_t)nb * BRICK * sizeof(uint16_t));
        if (!d_frac || !d_cell || !d_k0 || !d_span || !d_info) return fail(v, TSDF_ERR_OOM, "colour axis tables");
        cudaError_t e = cudaMemcpy(d_frac, frac.data(), nc * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_cell, cell.data(), nc, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_k0, k0.data(), (nb + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_span, span.data(), (size_t)nb * BRICK * sizeof(uint16_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_info, info.data(), nb * sizeof(uint16_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(v, e, "colour axis tables");
        v->vol.tab.frac[a] = d_frac;
        v->vol.tab.cell[a] = d_cell;
        v->vol.tab.k0[a] = d_k0;
        v->vol.tab.span[a] = d_span;
        v->vol.tab.info[a] = d_info;
    }
    return TSDF_OK;
}

tsdf_status tsdf_create_ex(const int32_t dims_geo[3], const int32_t dims_col[3], float voxel_size, float mu,
                           int32_t max_weight, const tsdf_params* params, tsdf_volume** out) {
    if (!out || !dims_geo || !dims_col) return TSDF_ERR_INVALID_ARG;
    *out = nullptr;
    tsdf_params p;
    tsdf_params_default(&p);
    if (params) p = *params;
    for (int a = 0; a < 3; ++a) {
        if (dims_geo[a] < 1 || dims_geo[a] > MAX_DIM || dims_col[a] < 1 || dims_col[a] > MAX_DIM)
            return TSDF_ERR_INVALID_ARG;
        if ((int64_t)dims_col[a] * dims_geo[0] != (int64_t)dims_col[0] * dims_geo[a]) return TSDF_ERR_INVALID_ARG;
        if (dims_col[a] > 8 * dims_geo[a]) return TSDF_ERR_INVALID_ARG;  // colour/geometry ratio <= 8
    }
    // z-slab: [z0, z1) of the geometry, cut at whole colour voxels
    const bool slab = p.slab_z[0] != 0 || p.slab_z[1] != 0;
    const int32_t z0 = slab ? p.slab_z[0] : 0, z1 = slab ? p.slab_z[1] : dims_geo[2];
    if (slab && (z0 < 0 || z1 <= z0 || z1 > dims_geo[2] || ((int64_t)z0 * dims_col[2]) % dims_geo[2] != 0 ||
                 ((int64_t)z1 * dims_col[2]) % dims_geo[2] != 0))
        return TSDF_ERR_INVALID_ARG;
    if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size) || !(mu > 0.0f) || !std::isfinite(mu))
        return TSDF_ERR_INVALID_ARG;
    if (max_weight < 1 || max_weight > 255) return TSDF_ERR_INVALID_ARG;
    if (!(p.sigma > 0.0f) || !std::isfinite(p.sigma)) return TSDF_ERR_INVALID_ARG;
    if (p.colour_mode < 0 || p.colour_mode > 1 || p.sample_mode < 0 || p.sample_mode > 1) return TSDF_ERR_INVALID_ARG;
    tsdf_volume* v = new (std::nothrow) tsdf_volume();
    if (v) v->prof_mask = (1u << TSDF_PHASE_COUNT) - 1u;
    if (!v) return TSDF_ERR_OOM;
    v->stream = (cudaStream_t)p.stream;
    v->alloc = p.allocator;
    if ((v->alloc.alloc == nullptr) != (v->alloc.free == nullptr)) {
        delete v;
        return TSDF_ERR_INVALID_ARG;
    }
    v->ngz_all = dims_geo[2];
    v->ncz_all = dims_col[2];
    v->slab_z0 = z0;
    v->slab_z1 = z1;
    // held z ranges: the slab's colour slice and its geometry widened by the
    // voxel on each side that the band gate's trilinear corners reach
    v->zoff_g = slab ? std::max(0, z0 - 1) : 0;
    v->zoff_c = (int32_t)((int64_t)z0 * dims_col[2] / dims_geo[2]);
    for (int a = 0; a < 3; ++a) {
        v->ng[a] = dims_geo[a];
        v->nc[a] = dims_col[a];
    }
    if (slab) {
        v->ng[2] = std::min(dims_geo[2], z1 + 1) - v->zoff_g;
        v->nc[2] = (int32_t)((int64_t)z1 * dims_col[2] / dims_geo[2]) - v->zoff_c;
    }
    for (int a = 0; a < 3; ++a) {
        v->nb[a] = (v->ng[a] + BRICK - 1) / BRICK;
        v->ncb[a] = (v->nc[a] + BRICK - 1) / BRICK;
    }
    v->s_g = voxel_size;
    v->s_c = (float)((double)dims_geo[0] * (double)voxel_size / (double)dims_col[0]);
    for (int a = 0; a < 3; ++a)
        v->origin[a] = std::isnan(p.origin[a]) ? (float)(-0.5 * (double)dims_geo[a] * (double)voxel_size) : p.origin[a];
    // the volumes must lie within 10^6 m of the world origin (every voxel's
    // camera depth then stays far inside the range where the projection's
    // reciprocal is exact)
    bool bounded = finite_all(v->origin, 3);
    for (int a = 0; a < 3 && bounded; ++a)
        bounded = std::fabs((double)v->origin[a]) + (double)dims_geo[a] * (double)voxel_size <= MAX_COORD;
    if (!bounded) {
        delete v;
        return TSDF_ERR_INVALID_ARG;
    }
    v->mu = mu;
    v->sigma = p.sigma;
    v->band = std::isnan(p.band) ? v->s_c / mu : p.band;
    if (!(v->band >= 0.0f) || !std::isfinite(v->band)) {
        delete v;
        return TSDF_ERR_INVALID_ARG;
    }
    v->max_weight = max_weight;
    v->colour_mode = p.colour_mode;
    v->sample_mode = p.sample_mode;
    v->culling = p.culling ? 1 : 0;
    v->free_space = p.update_free_space ? 1 : 0;

    cudaError_t e = cudaGetDevice(&v->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete v;
        return TSDF_ERR_CUDA;
    }
    // the side stream takes the device's highest priority: the next frame's
    // depth tiles and brick culling then get the SM room that the current
    // frame's band kernel leaves, ahead of the colour-voxel kernel queued
    // behind it, and finish before that kernel does instead of after it
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) prio_greatest = 0;
    if (cudaStreamCreateWithPriority(&v->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->list_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->bricks_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->main_tail, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->frame_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->frame_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->upload_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&v->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->stats_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->stats_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->stats_ev_side[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->stats_ev_side[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&v->stats_host, 4 * sizeof(Counters)) != cudaSuccess) {
        cudaGetLastError();
        tsdf_destroy(v);
        return TSDF_ERR_CUDA;
    }
    std::memset(v->stats_host, 0, 4 * sizeof(Counters));
    v->grids.geo = sms * geometry_blocks_per_sm();
    v->grids.col = sms * colour_blocks_per_sm();
    v->grids.vox = sms * voxel_blocks_per_sm();
    v->grids.fuse = sms * fused_blocks_per_sm();

    const int64_t nbt = (int64_t)v->nb[0] * v->nb[1] * v->nb[2];
    const int64_t ncbt = (int64_t)v->ncb[0] * v->ncb[1] * v->ncb[2];
    const size_t need = (size_t)nbt * BRICK_VOX * 5 + (size_t)ncbt * BRICK_VOX * 4 + (size_t)nbt * (sizeof(BrickSummary) + 25) +
                        (size_t)vox_capacity(nbt) * sizeof(uint2);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need > free_b) {
        delete v;
        return TSDF_ERR_OOM;
    }
    cudaGetLastError();
    v->vol.F = (float*)dev_alloc(v, (size_t)nbt * BRICK_VOX * sizeof(float));
    v->vol.W = (uint8_t*)dev_alloc(v, (size_t)nbt * BRICK_VOX);
    v->vol.C = (uint32_t*)dev_alloc(v, (size_t)ncbt * BRICK_VOX * sizeof(uint32_t));
    v->vol.summ = (BrickSummary*)dev_alloc(v, (size_t)nbt * sizeof(BrickSummary));
    v->scr.ctr = (Counters*)dev_alloc(v, sizeof(Counters));
    v->scr.geo_list = (uint32_t*)dev_alloc(v, (size_t)nbt * sizeof(uint32_t));
    v->scr.vis_list = (uint32_t*)dev_alloc(v, (size_t)nbt * sizeof(uint32_t));
    v->scr.col_list = (uint32_t*)dev_alloc(v, (size_t)nbt * sizeof(uint32_t));
    v->scr.col_act = (uint8_t*)dev_alloc(v, (size_t)nbt);
    v->scr.err = (uint32_t*)dev_alloc(v, sizeof(uint32_t));
    // fused frame: per-brick state bytes and neighbour counts, the ready queue and its counters
    v->scr.bstate = (uint8_t*)dev_alloc(v, (size_t)nbt);
    v->scr.need = (uint32_t*)dev_alloc(v, (size_t)nbt * sizeof(uint32_t));
    v->scr.ready = (unsigned long long*)dev_alloc(v, (size_t)nbt * sizeof(unsigned long long));
    v->scr.fsync = (FuseSync*)dev_alloc(v, sizeof(FuseSync));
    // band-gate voxel records of one frame; records that do not fit are
    // finished by the band kernel itself, so the capacity only bounds memory
    v->scr.vox_cap = (uint32_t)vox_capacity(nbt);
    if (const char* cap = std::getenv("TSDF_VOXEL_RECORD_CAPACITY")) {  // test / tuning override
        const long long n = std::atoll(cap);
        if (n >= 1 && n < (long long)v->scr.vox_cap) v->scr.vox_cap = (uint32_t)n;
    }
    v->scr.vox = (uint2*)dev_alloc(v, (size_t)v->scr.vox_cap * sizeof(uint2));
    if (!v->vol.F || !v->vol.W || !v->vol.C || !v->vol.summ || !v->scr.ctr || !v->scr.geo_list || !v->scr.vis_list ||
        !v->scr.col_list || !v->scr.col_act || !v->scr.err || !v->scr.vox || !v->scr.bstate || !v->scr.need || !v->scr.ready ||
        !v->scr.fsync) {
        tsdf_destroy(v);
        return TSDF_ERR_OOM;
    }
    {
        const tsdf_status ts = build_axis_tables(v);
        if (ts != TSDF_OK) {
            tsdf_destroy(v);
            return ts;
        }
    }
    e = cudaMemsetAsync(v->vol.F, 0, (size_t)nbt * BRICK_VOX * sizeof(float), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->vol.W, 0, (size_t)nbt * BRICK_VOX, v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->vol.C, 0, (size_t)ncbt * BRICK_VOX * sizeof(uint32_t), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->scr.ctr, 0, sizeof(Counters), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->scr.err, 0, sizeof(uint32_t), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->scr.ready, 0, (size_t)nbt * sizeof(unsigned long long), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->scr.fsync, 0, sizeof(FuseSync), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->scr.col_act, 0, (size_t)nbt, v->stream);
    if (e == cudaSuccess) e = launch_init_summaries(v->vol.summ, nbt, v->stream);
    if (e != cudaSuccess) {
        tsdf_destroy(v);
        return TSDF_ERR_CUDA;
    }
    *out = v;
    return TSDF_OK;
}

tsdf_status tsdf_create(const int32_t dims_geo[3], const int32_t dims_col[3], float voxel_size, float mu,
                        int32_t max_weight, tsdf_volume** out) {
    return tsdf_create_ex(dims_geo, dims_col, voxel_size, mu, max_weight, nullptr, out);
}

void tsdf_destroy(tsdf_volume* v) {
    if (!v) return;
    cudaStreamSynchronize(v->stream);
    if (v->side) {
        cudaStreamSynchronize(v->side);
        cudaStreamDestroy(v->side);
    }
    if (v->copy) {
        cudaStreamSynchronize(v->copy);
        cudaStreamDestroy(v->copy);
    }
    for (cudaEvent_t x : {v->list_done, v->bricks_done, v->main_tail, v->frame_done[0], v->frame_done[1], v->upload_done,
                          v->stats_ev[0], v->stats_ev[1],
                          v->stats_ev_side[0], v->stats_ev_side[1]})
        if (x) cudaEventDestroy(x);
    if (v->stats_host) cudaFreeHost(v->stats_host);
    for (auto* list : {&v->ev_pending, &v->ev_pool})
        for (auto& es : *list)
            for (auto& x : es.e) cudaEventDestroy(x);
    while (!v->blocks.empty()) dev_free(v, v->blocks.back().p);
    cudaGetLastError();
    delete v;
}

tsdf_status tsdf_set_stream(tsdf_volume* v, void* stream) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    cudaStreamSynchronize(v->stream);
    v->stream = (cudaStream_t)stream;
    v->chain_ok = false;
    return TSDF_OK;
}

tsdf_status tsdf_integrate(tsdf_volume* v, const uint16_t* depth_mm, tsdf_image_size dsz, const uint8_t* rgb_hwc,
                           tsdf_image_size csz, const float K_depth[9], const float K_rgb[9],
                           const float T_world_depth[16], const float T_depth_rgb[16]) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (!depth_mm || !rgb_hwc || !K_depth || !K_rgb || !T_world_depth || !T_depth_rgb)
        return fail(v, TSDF_ERR_INVALID_ARG, "NULL argument");
    if (dsz.width < 1 || dsz.height < 1 || csz.width < 1 || csz.height < 1 || dsz.width > MAX_IMAGE ||
        dsz.height > MAX_IMAGE || csz.width > MAX_IMAGE || csz.height > MAX_IMAGE)
        return fail(v, TSDF_ERR_INVALID_ARG, "image size outside 1..16384");
    float Kdi[9], Kri[9];
    if (!finite_all(K_depth, 9) || !finite_all(K_rgb, 9) || !invert3(K_depth, Kdi) || !invert3(K_rgb, Kri))
        return fail(v, TSDF_ERR_INVALID_ARG, "intrinsics not finite or singular");
    if (!rigid_ok(T_world_depth) || !rigid_ok(T_depth_rgb))
        return fail(v, TSDF_ERR_INVALID_ARG, "transform not finite or not rigid");
    if (!translation_ok(T_world_depth) || !translation_ok(T_depth_rgb))
        return fail(v, TSDF_ERR_INVALID_ARG, "translation beyond 10^6 m");

    FrameConst c;
    frame_constants(v, K_depth, K_rgb, T_world_depth, T_depth_rgb, dsz.width, dsz.height, csz.width, csz.height, c);
    c.frame_tag = (uint32_t)(v->frames % 0xFFFFFFFFll) + 1u;  // never 0 (the queue's initial value)
    c.fused = v->schedule == TSDF_SCHEDULE_FUSED && c.kd_pinhole ? 1 : 0;

    const size_t dbytes = (size_t)dsz.width * dsz.height * sizeof(uint16_t);
    const size_t cbytes = (size_t)csz.width * csz.height * 3;
    const uint16_t* d_depth = depth_mm;
    const uint8_t* d_rgb = rgb_hwc;
    cudaError_t e = cudaSuccess;
    tsdf_volume::EventSet* evs = nullptr;
    if (v->profiling) {
        if (v->ev_pool.empty()) {
            tsdf_volume::EventSet es;
            for (auto& x : es.e)
                if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(v, e, "profiling events");
            v->ev_pool.push_back(es);
        }
        v->ev_pending.push_back(v->ev_pool.back());
        v->ev_pool.pop_back();
        evs = &v->ev_pending.back();
        if (v->prof_mask & 1u) cudaEventRecord(evs->e[0], v->stream);
    }
    // Frame pipelining (see tsdf_volume::side): depth tiles and brick
    // culling go to the side stream, which waits for the previous frame's
    // colour list; the geometry update waits for them.  Host frames are
    // uploaded on the copy stream once the frame before the previous one (the
    // last user of their staging half) is done.  Timing of the first three
    // phases needs them in stream order, so it turns this off.
    const bool pipe = !(v->profiling && (v->prof_mask & 0x7u));
    // a device depth image is read by the side stream: unless the caller
    // declared its device images complete at the call, the side stream waits
    // for all the work queued on the handle's stream before it
    const bool chained = pipe && v->chain_ok && !(is_device_ptr(depth_mm) && !v->inputs_ready);
    cudaStream_t pre = pipe ? v->side : v->stream;
    cudaStream_t up = chained ? v->copy : pre;  // the stream of the host uploads
    if (pipe) {
        if (chained) {
            e = cudaStreamWaitEvent(v->copy, v->frame_done[v->frames & 1], 0);
        } else {
            e = cudaEventRecord(v->main_tail, v->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(v->side, v->main_tail, 0);
        }
        if (e != cudaSuccess) return cuda_fail(v, e, "frame pipeline");
    }
    if (!is_device_ptr(depth_mm)) {
        // host frames alternate between two staging buffers, since the colour
        // kernels of the previous frame may still read the other one
        const bool second = pipe && (v->frames & 1);
        uint16_t*& buf = second ? v->d_depth2 : v->d_depth;
        size_t& cap = second ? v->d_depth2_cap : v->d_depth_cap;
        if (cap < dbytes) {
            dev_free(v, buf);
            buf = (uint16_t*)dev_alloc(v, dbytes);
            cap = buf ? dbytes : 0;
            if (!buf) return fail(v, TSDF_ERR_OOM, "depth staging buffer");
        }
        e = cudaMemcpyAsync(buf, depth_mm, dbytes, cudaMemcpyHostToDevice, up);
        if (e != cudaSuccess) return cuda_fail(v, e, "depth upload");
        d_depth = buf;
    }
    if (!is_device_ptr(rgb_hwc)) {  // likewise for the RGB frame
        const bool second = pipe && (v->frames & 1);
        uint8_t*& buf = second ? v->d_rgb2 : v->d_rgb;
        size_t& cap = second ? v->d_rgb2_cap : v->d_rgb_cap;
        if (cap < cbytes) {
            dev_free(v, buf);
            buf = (uint8_t*)dev_alloc(v, cbytes);
            cap = buf ? cbytes : 0;
            if (!buf) return fail(v, TSDF_ERR_OOM, "RGB staging buffer");
        }
        e = cudaMemcpyAsync(buf, rgb_hwc, cbytes, cudaMemcpyHostToDevice, up);
        if (e != cudaSuccess) return cuda_fail(v, e, "RGB upload");
        d_rgb = buf;
    }
    if (chained) {
        // the depth tiles read the upload, and they and the culling overwrite
        // what the previous frame's colour list reads
        e = cudaEventRecord(v->upload_done, v->copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->side, v->upload_done, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->side, v->list_done, 0);
        if (e != cudaSuccess) return cuda_fail(v, e, "frame pipeline");
    }
    if (pipe && v->stats_pending) {
        // a counter read queued since the last frame must finish before the
        // depth tiles reset the geometry-side counters (the uploads above
        // need not wait for it)
        e = cudaStreamWaitEvent(v->side, v->stats_last, 0);
        if (e != cudaSuccess) return cuda_fail(v, e, "frame pipeline");
    }
    v->stats_pending = false;
    const tsdf_status ds = depth_scratch(v, (size_t)c.tiles_x * c.tiles_y, dsz);
    if (ds != TSDF_OK) return ds;
    // boundary k + 1 (after phase k, before phase k + 1) is recorded when either side is timed
    cudaEvent_t marks[TSDF_PHASE_COUNT];
    for (int k = 0; k < TSDF_PHASE_COUNT; ++k)
        marks[k] = (evs && (v->prof_mask & (3u << k))) ? evs->e[k + 1] : nullptr;
    e = launch_frame_pre(c, v->vol, v->scr, d_depth, pre, evs && !pipe ? marks : nullptr);
    if (e != cudaSuccess) return cuda_fail(v, e, "integrate launch");
    if (pipe) {
        e = cudaEventRecord(v->bricks_done, v->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->stream, v->bricks_done, 0);
        if (e != cudaSuccess) return cuda_fail(v, e, "frame pipeline");
        if (marks[2]) cudaEventRecord(marks[2], v->stream);  // the geometry update starts here
    }
    e = launch_frame_post(c, v->vol, v->scr, d_depth, d_rgb, v->grids, v->stream, evs ? marks : nullptr,
                          pipe ? v->list_done : nullptr);
    if (e == cudaSuccess && pipe) e = cudaEventRecord(v->frame_done[v->frames & 1], v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "integrate launch");
    v->chain_ok = pipe;
    ++v->frames;
    return TSDF_OK;
}

tsdf_status tsdf_set_frame_schedule(tsdf_volume* v, int32_t schedule) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (schedule != TSDF_SCHEDULE_KERNELS && schedule != TSDF_SCHEDULE_FUSED)
        return fail(v, TSDF_ERR_INVALID_ARG, "frame schedule: TSDF_SCHEDULE_KERNELS or TSDF_SCHEDULE_FUSED");
    v->schedule = schedule;
    return TSDF_OK;
}

tsdf_status tsdf_set_device_inputs_ready(tsdf_volume* v, int32_t ready) {
    if (!v || (ready != 0 && ready != 1)) return TSDF_ERR_INVALID_ARG;
    v->inputs_ready = ready != 0;
    return TSDF_OK;
}

tsdf_status tsdf_get_frame_schedule(const tsdf_volume* v, int32_t* schedule) {
    if (!v || !schedule) return TSDF_ERR_INVALID_ARG;
    *schedule = v->schedule;
    return TSDF_OK;
}

tsdf_status tsdf_fused_inject_stall(tsdf_volume* v) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    const unsigned one = 1u;
    cudaError_t e = cudaMemcpyAsync(&v->scr.fsync->stall, &one, sizeof one, cudaMemcpyHostToDevice, v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "stall injection");
}

tsdf_status tsdf_synchronize(tsdf_volume* v) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    return check_device_error(v);
}

tsdf_status tsdf_read(tsdf_volume* v, float* tsdf, uint8_t* w_geo, uint32_t* rgbw) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    tsdf_status s = read_volume<float>(v, v->vol.F, tsdf, v->ng, launch_to_linear_f32);
    if (s == TSDF_OK) s = read_volume<uint8_t>(v, v->vol.W, w_geo, v->ng, launch_to_linear_u8);
    if (s == TSDF_OK) s = read_volume<uint32_t>(v, v->vol.C, rgbw, v->nc, launch_to_linear_u32);
    if (s != TSDF_OK) return s;
    return check_device_error(v);
}

tsdf_status tsdf_write(tsdf_volume* v, const float* tsdf, const uint8_t* w_geo, const uint32_t* rgbw) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    v->chain_ok = false;
    tsdf_status s = write_volume<float>(v, v->vol.F, tsdf, v->ng, launch_from_linear_f32);
    if (s == TSDF_OK) s = write_volume<uint8_t>(v, v->vol.W, w_geo, v->ng, launch_from_linear_u8);
    if (s == TSDF_OK) s = write_volume<uint32_t>(v, v->vol.C, rgbw, v->nc, launch_from_linear_u32);
    if (s != TSDF_OK) return s;
    cudaError_t e = launch_recompute_summaries(v->vol.F, v->vol.W, v->vol.summ, v->ng, v->band, v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "summaries");
    return check_device_error(v);
}

tsdf_status tsdf_get_info(const tsdf_volume* v, tsdf_info* o) {
    if (!v || !o) return TSDF_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof *o);
    for (int a = 0; a < 3; ++a) {
        o->dims_geo[a] = v->ng[a];
        o->dims_col[a] = v->nc[a];
        o->origin[a] = v->origin[a];
    }
    o->voxel_geo = v->s_g;
    o->voxel_col = v->s_c;
    o->mu = v->mu;
    o->sigma = v->sigma;
    o->band = v->band;
    o->max_weight = v->max_weight;
    o->colour_mode = v->colour_mode;
    o->sample_mode = v->sample_mode;
    o->culling = v->culling;
    o->update_free_space = v->free_space;
    o->frames = v->frames;
    o->device_bytes = v->device_bytes;
    o->dims_geo[2] = v->ngz_all;  // the whole volume's dims
    o->dims_col[2] = v->ncz_all;
    o->slab_z[0] = v->slab_z0;
    o->slab_z[1] = v->slab_z1;
    o->held_geo_z[0] = v->zoff_g;
    o->held_geo_z[1] = v->zoff_g + v->ng[2];
    o->held_col_z[0] = v->zoff_c;
    o->held_col_z[1] = v->zoff_c + v->nc[2];
    return TSDF_OK;
}

static_assert(sizeof(Counters) == TSDF_STATS_COPY_BYTES, "the header states the size of one counter read");

static void fill_stats(const tsdf_volume* v, const Counters& h, tsdf_stats* o) {
    o->geo_updated = (int64_t)h.geo_updated;
    o->col_updated = (int64_t)h.col_updated;
    o->geo_bricks = h.n_geo;
    o->col_bricks = h.n_col + h.n_col_light;
    o->visible_bricks = h.n_vis;
    o->total_bricks = (int64_t)v->nb[0] * v->nb[1] * v->nb[2];
    o->frames_counted = (int64_t)h.frames;
    o->total_geo_updated = (int64_t)(h.tot_geo_updated + h.geo_updated);
    o->total_col_updated = (int64_t)(h.tot_col_updated + h.col_updated);
    o->total_geo_bricks = (int64_t)(h.tot_geo_bricks + h.n_geo);
    o->total_col_bricks = (int64_t)(h.tot_col_bricks + h.n_col + h.n_col_light);
    o->total_visible_bricks = (int64_t)(h.tot_vis_bricks + h.n_vis);
    o->total_col_active_bricks = (int64_t)(h.tot_col_active + h.n_col_active);
    o->total_cells = (int64_t)(h.tot_cells + h.n_cells);
    o->total_geo_changed_bricks = (int64_t)(h.tot_geo_changed + h.n_geo_changed);
}

tsdf_status tsdf_get_stats(tsdf_volume* v, tsdf_stats* o) {
    if (!v || !o) return TSDF_ERR_INVALID_ARG;
    Counters h;
    cudaError_t e = cudaMemcpyAsync(&h, v->scr.ctr, sizeof h, cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "stats read");
    fill_stats(v, h, o);
    return TSDF_OK;
}

tsdf_status tsdf_stats_request(tsdf_volume* v, int32_t slot) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (slot != 0 && slot != 1) return fail(v, TSDF_ERR_INVALID_ARG, "stats slot must be 0 or 1");
    Counters* h = v->stats_host + 2 * slot;
    cudaError_t e = cudaSuccess;
    // after a pipelined frame, the geometry-side counters are copied on the
    // side stream once the frame's colour list is done, ahead of the next
    // frame's depth tiles (see tsdf_volume::stats_host)
    const bool split = v->chain_ok;
    if (split) {
        e = cudaStreamWaitEvent(v->side, v->list_done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h + 1, v->scr.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, v->side);
        if (e == cudaSuccess) e = cudaEventRecord(v->stats_ev_side[slot], v->side);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, v->scr.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess) e = cudaEventRecord(v->stats_ev[slot], v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "stats request");
    v->stats_split[slot] = split;
    if (!split) {
        v->stats_last = v->stats_ev[slot];
        v->stats_pending = true;
    }
    return TSDF_OK;
}

tsdf_status tsdf_stats_collect(tsdf_volume* v, int32_t slot, tsdf_stats* o) {
    if (!v || !o) return TSDF_ERR_INVALID_ARG;
    if (slot != 0 && slot != 1) return fail(v, TSDF_ERR_INVALID_ARG, "stats slot must be 0 or 1");
    cudaError_t e = cudaEventSynchronize(v->stats_ev[slot]);
    if (e == cudaSuccess && v->stats_split[slot]) e = cudaEventSynchronize(v->stats_ev_side[slot]);
    if (e != cudaSuccess) return cuda_fail(v, e, "stats collect");
    Counters h = v->stats_host[2 * slot];
    if (v->stats_split[slot]) {  // the geometry-side counters (those k_depth_tiles folds and resets)
        const Counters& g = v->stats_host[2 * slot + 1];
        h.n_geo = g.n_geo;
        h.n_vis = g.n_vis;
        h.geo_next = g.geo_next;
        h.n_geo_changed = g.n_geo_changed;
        h.geo_updated = g.geo_updated;
        h.frames = g.frames;
        h.tot_geo_updated = g.tot_geo_updated;
        h.tot_geo_bricks = g.tot_geo_bricks;
        h.tot_vis_bricks = g.tot_vis_bricks;
        h.tot_geo_changed = g.tot_geo_changed;
    }
    fill_stats(v, h, o);
    return TSDF_OK;
}

static tsdf_status drain_profile(tsdf_volume* v) {
    cudaError_t e = cudaStreamSynchronize(v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "profile sync");
    for (auto& es : v->ev_pending) {
        for (int k = 0; k < TSDF_PHASE_COUNT; ++k) {
            float ms = 0.0f;
            if ((v->prof_mask >> k) & 1u)
                if (cudaEventElapsedTime(&ms, es.e[k], es.e[k + 1]) == cudaSuccess) v->prof_ms[k] += ms;
        }
        ++v->prof_frames;
        v->ev_pool.push_back(es);
    }
    v->ev_pending.clear();
    cudaGetLastError();
    return TSDF_OK;
}

tsdf_status tsdf_profile_enable(tsdf_volume* v, int32_t enable) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    v->chain_ok = false;
    tsdf_status s = drain_profile(v);
    if (s != TSDF_OK) return s;
    v->profiling = enable != 0;
    for (double& x : v->prof_ms) x = 0.0;
    v->prof_frames = 0;
    cudaError_t e = cudaMemsetAsync(v->scr.ctr, 0, sizeof(Counters), v->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "counter reset");
}

tsdf_status tsdf_profile_phases(tsdf_volume* v, uint32_t mask) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    v->chain_ok = false;
    if (mask == 0u || mask >= (1u << TSDF_PHASE_COUNT))
        return fail(v, TSDF_ERR_INVALID_ARG, "profile: phase mask outside 1 .. 2^7 - 1");
    tsdf_status s = drain_profile(v);
    if (s != TSDF_OK) return s;
    v->prof_mask = mask;
    for (double& x : v->prof_ms) x = 0.0;
    v->prof_frames = 0;
    return TSDF_OK;
}

tsdf_status tsdf_profile_read(tsdf_volume* v, tsdf_profile_report* out) {
    if (!v || !out) return TSDF_ERR_INVALID_ARG;
    tsdf_status s = drain_profile(v);
    if (s != TSDF_OK) return s;
    out->frames = v->prof_frames;
    for (int k = 0; k < TSDF_PHASE_COUNT; ++k) out->ms[k] = v->prof_ms[k];
    return TSDF_OK;
}

// ------------------------------------------------------------- checkpoint --
namespace {
struct FileHeader {
    char magic[8];
    uint32_t version;
    int32_t dims_geo[3], dims_col[3];
    float voxel, mu, origin[3], sigma, band;
    int32_t max_weight, colour_mode, sample_mode, free_space;
    int64_t frames;
    int32_t zoff_g, zoff_c;  // version 2: global z index of held geometry / colour z = 0
};
}  // namespace

tsdf_status tsdf_save(tsdf_volume* v, const char* path) {
    if (!v || !path) return TSDF_ERR_INVALID_ARG;
    const size_t ng = (size_t)v->ng[0] * v->ng[1] * v->ng[2];
    const size_t nc = (size_t)v->nc[0] * v->nc[1] * v->nc[2];
    std::vector<float> F(ng);
    std::vector<uint8_t> W(ng);
    std::vector<uint32_t> C(nc);
    tsdf_status s = tsdf_read(v, F.data(), W.data(), C.data());
    if (s != TSDF_OK) return s;
    FileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "TSDFVOL1", 8);
    h.version = 2;
    h.zoff_g = v->zoff_g;
    h.zoff_c = v->zoff_c;
    for (int a = 0; a < 3; ++a) {
        h.dims_geo[a] = v->ng[a];
        h.dims_col[a] = v->nc[a];
        h.origin[a] = v->origin[a];
    }
    h.voxel = v->s_g;
    h.mu = v->mu;
    h.sigma = v->sigma;
    h.band = v->band;
    h.max_weight = v->max_weight;
    h.colour_mode = v->colour_mode;
    h.sample_mode = v->sample_mode;
    h.free_space = v->free_space;
    h.frames = v->frames;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(v, TSDF_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(F.data(), sizeof(float), ng, f) == ng &&
              std::fwrite(W.data(), 1, ng, f) == ng && std::fwrite(C.data(), sizeof(uint32_t), nc, f) == nc;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TSDF_OK : fail(v, TSDF_ERR_IO, std::string("write failed: ") + path);
}

tsdf_status tsdf_load(tsdf_volume* v, const char* path) {
    if (!v || !path) return TSDF_ERR_INVALID_ARG;
    v->chain_ok = false;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(v, TSDF_ERR_IO, std::string("cannot open ") + path);
    FileHeader h;
    if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, "TSDFVOL1", 8) != 0 || h.version != 2) {
        std::fclose(f);
        return fail(v, TSDF_ERR_IO, "not a TSDFVOL1 version 2 checkpoint");
    }
    if (h.zoff_g != v->zoff_g || h.zoff_c != v->zoff_c) {
        std::fclose(f);
        return fail(v, TSDF_ERR_INVALID_ARG, "checkpoint holds another z-slab");
    }
    for (int a = 0; a < 3; ++a)
        if (h.dims_geo[a] != v->ng[a] || h.dims_col[a] != v->nc[a]) {
            std::fclose(f);
            return fail(v, TSDF_ERR_INVALID_ARG, "checkpoint dims differ from the handle's");
        }
    const size_t ng = (size_t)v->ng[0] * v->ng[1] * v->ng[2];
    const size_t nc = (size_t)v->nc[0] * v->nc[1] * v->nc[2];
    std::vector<float> F(ng);
    std::vector<uint8_t> W(ng);
    std::vector<uint32_t> C(nc);
    bool ok = std::fread(F.data(), sizeof(float), ng, f) == ng && std::fread(W.data(), 1, ng, f) == ng &&
              std::fread(C.data(), sizeof(uint32_t), nc, f) == nc;
    std::fclose(f);
    if (!ok) return fail(v, TSDF_ERR_IO, "truncated checkpoint");
    tsdf_status s = tsdf_write(v, F.data(), W.data(), C.data());
    if (s == TSDF_OK) v->frames = h.frames;
    return s;
}

}  // extern "C"
