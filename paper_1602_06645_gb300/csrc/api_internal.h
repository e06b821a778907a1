// Host-side internals shared by the C-ABI translation units: the handle
// structure and the validation / allocation helpers of tsdf_api.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/tsdf.h"
#include "common.cuh"

using tsdf::LaunchGrids;
using tsdf::Scratch;
using tsdf::Volumes;

struct tsdf_volume {
    int32_t ng[3], nc[3], nb[3], ncb[3];  // held voxels and bricks per axis
    // z-slab handles: the whole volume's z dims, the slab [slab_z0, slab_z1)
    // and the global z index of held geometry / colour z = 0 (whole: 0, 0)
    int32_t ngz_all, ncz_all, slab_z0, slab_z1, zoff_g, zoff_c;
    float s_g, s_c, origin[3], mu, sigma, band;
    int32_t max_weight, colour_mode, sample_mode, culling, free_space;
    cudaStream_t stream;
    tsdf_allocator alloc;
    int device;
    LaunchGrids grids;
    Volumes vol;
    Scratch scr;
    uint32_t* depth_tiles;
    size_t depth_tiles_cap;
    uint16_t* d_depth;
    size_t d_depth_cap;
    // Frame pipelining: the depth tiles and brick culling of frame k + 1 run on
    // `side` while frame k's colour kernels finish on `stream`.  list_done is
    // recorded on `stream` after frame k's colour list; bricks_done on `side`
    // after frame k + 1's culling.  chain_ok: the last call that touched the
    // volume on `stream` was a pipelined tsdf_integrate (else `side` waits for
    // all of `stream` first).  Host depth frames alternate between two
    // staging buffers.  `side` has the device's highest stream priority, so
    // its small blocks are dispatched ahead of the colour kernel queued
    // (programmatic launch) behind frame k's band kernel.
    cudaStream_t side;
    cudaEvent_t list_done, bricks_done, main_tail;
    // frame_done[k & 1] is recorded on `stream` after pipelined frame k's
    // last kernel.  Frame k + 2's host frames are uploaded on `copy` into
    // the staging half frame k used, after frame_done[k & 1] only: the
    // uploads overlap frame k + 1's geometry update, and no counter read or
    // colour list queued on `side` holds them back; `side` waits for
    // upload_done before the depth tiles.
    cudaEvent_t frame_done[2], upload_done;
    cudaStream_t copy;
    bool chain_ok;
    // Asynchronous counter reads (tsdf_stats_request / tsdf_stats_collect):
    // per slot, page-locked copies of the counters taken on `stream` (entry
    // 2 slot) and, after a pipelined frame, on `side` (entry 2 slot + 1) with
    // their completion events.  The next frame's depth tiles, queued on `side`
    // behind the side copy, reset the geometry-side counters, so a split read
    // takes those from the side copy (made once the frame's colour list is
    // done) and the colour-side ones from the stream copy.  After a frame that
    // was not pipelined the read is one stream copy, and the next frame's depth
    // tiles wait for it (stats_pending).
    tsdf::Counters* stats_host;
    cudaEvent_t stats_ev[2], stats_ev_side[2];
    bool stats_split[2];
    cudaEvent_t stats_last;
    bool stats_pending;
    uint16_t* d_depth2;
    size_t d_depth2_cap;
    uint8_t* d_rgb2;
    size_t d_rgb2_cap;
    uint8_t* d_rgb;
    size_t d_rgb_cap;
    int64_t frames;
    int32_t schedule = TSDF_SCHEDULE_KERNELS;  // tsdf_set_frame_schedule
    bool inputs_ready = false;                 // tsdf_set_device_inputs_ready
    int64_t device_bytes;
    std::string last_error;
    // phase timing (tsdf_profile_enable)
    struct EventSet {
        cudaEvent_t e[TSDF_PHASE_COUNT + 1];
    };
    bool profiling;
    uint32_t prof_mask;  // phases timed (bit k = phase k)
    std::vector<EventSet> ev_pending, ev_pool;
    double prof_ms[TSDF_PHASE_COUNT];
    int64_t prof_frames;
    struct Block {
        void* p;
        size_t bytes;
    };
    std::vector<Block> blocks;
};


namespace tsdf_host {
tsdf_status fail(tsdf_volume* v, tsdf_status s, const std::string& msg);
tsdf_status cuda_fail(tsdf_volume* v, cudaError_t e, const char* where);
void* dev_alloc(tsdf_volume* v, size_t bytes);
void dev_free(tsdf_volume* v, void* p);
bool finite_all(const float* a, int n);
bool is_device_ptr(const void* p);
bool rigid_ok(const float T[16]);
constexpr double MAX_COORD = 1e6;  // metres: volume corners and camera translations stay within this
bool translation_ok(const float T[16]);
bool invert3(const float K[9], float out[9]);
void frame_constants(const tsdf_volume* v, const float Kd[9], const float Kr[9], const float Twd[16],
                     const float Tdr[16], int dw, int dh, int cw, int ch, tsdf::FrameConst& c);
tsdf_status check_device_error(tsdf_volume* v);
// Upload a frame's depth image (host or device) and size the depth-tile
// buffer; sets *d_depth to the device copy.
tsdf_status stage_depth(tsdf_volume* v, const uint16_t* depth_mm, tsdf_image_size dsz, int tiles,
                        const uint16_t** d_depth);
// The frame's depth-tile buffer: the 8x8 tiles, then (16-byte aligned) the
// depth in metres, W * H floats; grown when a larger frame arrives.
tsdf_status depth_scratch(tsdf_volume* v, size_t tiles, tsdf_image_size dsz);
// Validated ray-cast constants of a camera (as tsdf_raycast takes them).
tsdf_status raycast_constants(tsdf_volume* v, const float K[9], const float T_world_camera[16], tsdf_image_size size,
                              const tsdf_raycast_params* params, tsdf::RayConst& c);
}  // namespace tsdf_host
