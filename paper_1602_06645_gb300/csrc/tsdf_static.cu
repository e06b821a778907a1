// Allocation-free geometry fusion: tsdf_integrate_geometry_static.
//
// Some callers cannot allocate device memory at all: code that runs while
// another framework owns the device allocator (and must not call cudaMalloc
// behind its back), hosts with a fixed device-memory budget decided up front,
// or callers that only hand over buffers they already own.  This entry point
// needs no handle and allocates nothing: the caller passes the depth image and
// its own TSDF / weight arrays; the per-frame scratch (work counters, depth
// tiles, brick work list) lives in one file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/tsdf.h"
#include "api_internal.h"
#include "common.cuh"

using namespace tsdf;

namespace {

constexpr int64_t STATIC_MAX_BRICKS = TSDF_STATIC_MAX_BRICKS;   // 8^3 geometry bricks
constexpr int64_t STATIC_MAX_TILES = TSDF_STATIC_MAX_DEPTH_TILES;  // 8x8 depth tiles
constexpr size_t COUNTERS_BYTES = 256;
constexpr size_t TILES_BYTES = (size_t)STATIC_MAX_TILES * sizeof(uint32_t);
constexpr size_t LIST_BYTES = (size_t)STATIC_MAX_BRICKS * sizeof(uint32_t);
constexpr size_t SCRATCH_BYTES = COUNTERS_BYTES + TILES_BYTES + LIST_BYTES;
static_assert(SCRATCH_BYTES == TSDF_STATIC_SCRATCH_BYTES, "the header states the scratch size");
static_assert(sizeof(Counters) <= COUNTERS_BYTES, "counters do not fit their slot");

// The shared scratch.  In host code this name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_dev[MAX_DEVICES];  // device address of g_scratch per device, set on first use
int g_grid[MAX_DEVICES];

bool finite_n(const float* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

bool rigid(const float T[16]) {
    if (!finite_n(T, 16) || T[12] != 0.0f || T[13] != 0.0f || T[14] != 0.0f || T[15] != 1.0f) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += (double)T[k * 4 + i] * (double)T[k * 4 + j];
            if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-4) return false;
        }
    return true;
}

}  // namespace

extern "C" tsdf_status tsdf_integrate_geometry_static(const int32_t dims[3], float voxel_size, float mu,
                                                      int32_t max_weight, const float origin[3], float* tsdf_dev,
                                                      uint8_t* w_dev, const uint16_t* depth_dev, tsdf_image_size dsz,
                                                      const float K_depth[9], const float T_world_depth[16],
                                                      void* stream) {
    if (!dims || !origin || !tsdf_dev || !w_dev || !depth_dev || !K_depth || !T_world_depth)
        return TSDF_ERR_INVALID_ARG;
    // the three arrays must be device memory (a host array would be read and
    // written out of bounds by the kernels); this query allocates nothing
    if (!tsdf_host::is_device_ptr(tsdf_dev) || !tsdf_host::is_device_ptr(w_dev) ||
        !tsdf_host::is_device_ptr(depth_dev))
        return TSDF_ERR_INVALID_ARG;
    int64_t nbt = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > 4096) return TSDF_ERR_INVALID_ARG;
        nbt *= (dims[a] + BRICK - 1) / BRICK;
    }
    if (nbt > STATIC_MAX_BRICKS) return TSDF_ERR_INVALID_ARG;  // beyond the fixed scratch
    if (dsz.width < 1 || dsz.height < 1 || dsz.width > 16384 || dsz.height > 16384) return TSDF_ERR_INVALID_ARG;
    const int64_t tiles = (int64_t)((dsz.width + TILE_PX - 1) / TILE_PX) * ((dsz.height + TILE_PX - 1) / TILE_PX);
    if (tiles > STATIC_MAX_TILES) return TSDF_ERR_INVALID_ARG;
    if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size) || !(mu > 0.0f) || !std::isfinite(mu))
        return TSDF_ERR_INVALID_ARG;
    if (max_weight < 1 || max_weight > 255 || !finite_n(origin, 3) || !finite_n(K_depth, 9) || !rigid(T_world_depth))
        return TSDF_ERR_INVALID_ARG;
    {
        const double a = K_depth[0], b = K_depth[1], c = K_depth[2], d = K_depth[3], e = K_depth[4], f = K_depth[5],
                     g = K_depth[6], h = K_depth[7], i = K_depth[8];
        const double det = (a * (e * i - f * h) + b * (f * g - d * i)) + c * (d * h - e * g);
        if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return TSDF_ERR_INVALID_ARG;
    }

    // once per device, with that device current: the device address of the
    // scratch array and the persistent grid size.  The address belongs to the
    // device's primary context: after cudaDeviceReset the cached value is
    // stale, so the library must not be used across a device reset.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return TSDF_ERR_CUDA;
    }
    void* scratch = nullptr;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_dev[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TSDF_ERR_CUDA;
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return TSDF_ERR_CUDA;
            }
            g_grid[dev] = sms * geometry_linear_blocks_per_sm();
            g_scratch_dev[dev] = p;
        }
        scratch = g_scratch_dev[dev];
        grid = g_grid[dev];
    }
    unsigned char* base = static_cast<unsigned char*>(scratch);
    Counters* ctr = reinterpret_cast<Counters*>(base);  // zeroed by the first kernel of every call
    uint32_t* tile_buf = reinterpret_cast<uint32_t*>(base + COUNTERS_BYTES);
    uint32_t* list = reinterpret_cast<uint32_t*>(base + COUNTERS_BYTES + TILES_BYTES);

    VolumeDesc desc;
    for (int a = 0; a < 3; ++a) {
        desc.ng[a] = dims[a];
        desc.origin[a] = origin[a];
    }
    desc.s_g = voxel_size;
    desc.mu = mu;
    desc.max_weight = max_weight;
    FrameConst c;
    geometry_frame_constants(desc, K_depth, T_world_depth, dsz.width, dsz.height, c);
    cudaError_t e = launch_geometry_static(c, tsdf_dev, w_dev, depth_dev, ctr, tile_buf, list, grid,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    return TSDF_OK;
}
