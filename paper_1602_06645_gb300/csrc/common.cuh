// Internal declarations shared by the CUDA translation units of libtsdf.so.
//
// Numerics: every kernel is compiled with --fmad=false, so a product and a sum
// are rounded separately unless written as fmaf(); reciprocals, quotients and
// square roots use the correctly rounded __frcp_rn / __fdiv_rn / __fsqrt_rn.
// The operation order of each step is the one written in the comments; it is
// what makes the integer decisions (pixel choice, gates, weights and colours)
// reproducible bit for bit on any IEEE binary32 implementation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsdf {

// Volumes are stored brick-major: 8x8x8 voxel bricks, each brick contiguous
// (voxel (x,y,z) of a brick at ((z*8)+y)*8+x), bricks ordered x fastest.  A
// brick of F is 2 KB, of w 512 B, of colour 2 KB: whole DRAM sectors.
constexpr int BRICK = 8;
constexpr int BRICK_VOX = BRICK * BRICK * BRICK;
constexpr int TILE_PX = 8;         // depth-culling tiles are 8x8 pixels

// Per-frame constants, passed by value as a kernel parameter.
struct FrameConst {
    float R[9], t[3];      // world -> depth camera: the motion (R_n, t_n) of Eq. 5
    float Kd[9], Kdi[9];   // K_c and K_c^-1 (Eq. 6, Eq. 7)
    float Kr[9];           // K_hd (Eq. 4)
    float Rc[9], tc[3];    // (R_calib, t_calib), Eq. 3
    float origin[3];       // volume minimum corner (world)
    float s_g, s_c;        // geometry / colour voxel edge
    float inv_sg;          // 1/s_g (binary32 quotient)
    float mu, inv_mu;      // truncation distance and 1/mu
    float sigma2;          // sigma * sigma (Eq. 7)
    float band;            // TSDF band gate
    float cull_behind;     // metres beyond the farthest depth where nothing can change
    int32_t ng[3], nc[3];  // geometry / colour dims
    int32_t nb[3], ncb[3]; // bricks per axis (geometry / colour)
    int32_t dw, dh, cw, ch;
    int32_t tiles_x, tiles_y;
    int32_t kd_pinhole, kr_pinhole, kdi_pinhole;
    int32_t max_weight, free_space, sample_mode, colour_mode, culling;
    int32_t record_mode;   // 1: the band kernel only records (adjoint gate recording); no colour update
    int32_t zoff_g, zoff_c;  // z-slab: global z index of held geometry / colour z = 0 (whole volume: 0)
    uint32_t pix_bias;       // 0x4B000000 (dw + 1) mod 2^32: pixel index from the bits of u + 2^23, v + 2^23
    uint32_t frame_tag;      // nonzero, different in consecutive frames: marks this frame's ready-queue entries
    int32_t fused;           // 1: the frame runs as one fused launch (k_fused) instead of the kernel chain
};

// Min/max of F over observed voxels (w > 0) and min of w over the in-volume
// voxels of one geometry brick.  No observed voxel: fmin = +inf, fmax = -inf.
// flags: bit 0 / 1 = some observed voxel has F <= band + eps / F >= -band - eps;
// bits 2 + 2f / 3 + 2f = the same over face layer f (-x, +x, -y, +y, -z, +z).
struct BrickSummary {
    float fmin, fmax;
    uint32_t wmin;
    uint32_t flags;
};

// Band flags of one voxel at local brick position (x, y, z).
__host__ __device__ __forceinline__ uint32_t band_flags(bool observed, float f, float lo_thr, float hi_thr, int x,
                                                        int y, int z) {
    if (!observed) return 0u;
    const uint32_t b = (f <= lo_thr ? 1u : 0u) | (f >= hi_thr ? 2u : 0u);
    uint32_t m = b;
    if (x == 0) m |= b << 2;
    if (x == 7) m |= b << 4;
    if (y == 0) m |= b << 6;
    if (y == 7) m |= b << 8;
    if (z == 0) m |= b << 10;
    if (z == 7) m |= b << 12;
    return m;
}

struct Counters {
    uint32_t n_geo;      // geometry work list length
    uint32_t n_vis;      // visible brick list length
    uint32_t n_col;      // colour work list length
    uint32_t geo_next;   // persistent-loop work counters
    uint32_t col_next;
    uint32_t n_vox;      // band-gate voxel records (may exceed the buffer's capacity)
    uint32_t n_cells;    // trilinear cells that can pass the band gate
    uint32_t n_col_active;   // colour candidates with at least one such cell
    uint32_t n_geo_changed;  // geometry bricks with at least one updated voxel
    uint32_t n_col_light;    // colour work list entries filled from the buffer's end (taken last)
    unsigned long long geo_updated;
    unsigned long long col_updated;
    // running totals over frames, folded in by the first kernel of each frame
    unsigned long long frames;
    unsigned long long tot_geo_updated, tot_col_updated;
    unsigned long long tot_geo_bricks, tot_col_bricks, tot_vis_bricks;
    unsigned long long tot_cells, tot_col_active, tot_geo_changed;
};

// Device error word bits.
enum : uint32_t {
    ERR_TILE_RANGE = 1u,       // a colour voxel fell outside its brick's geometry tile
    ERR_RECORD_OVERFLOW = 2u,  // gate recording: band records exceeded their buffer
    ERR_PAIR_OVERFLOW = 4u,    // gate recording: (frame, voxel) pairs exceeded their buffer
    ERR_SLOT_OVERFLOW = 8u,    // adjoint: more distinct voxels or frames per voxel than reserved
    ERR_WAIT_TIMEOUT = 16u,    // fused frame: a bounded wait for ready colour work gave up
};

// Adjoint (photometric loss) buffers.
struct AdjFrame {  // world -> depth camera of one recorded frame (binary32 frame constants)
    float R[9], t[3];
};
struct AdjBuffers {
    uint32_t* pair_vox;     // linear colour index of each (frame, voxel) pair
    uint8_t* pair_frame;    // its frame
    uint32_t pair_cap;
    int32_t* slot_of;       // dense colour-volume map: slot of a voxel, -1 none
    uint32_t* V;            // voxel of each slot
    uint32_t* slot_count;   // frames per slot
    uint8_t* slot_frames;   // slot_cap x max_frames frame ids, ascending after finalize
    int32_t* n_valid;       // samples inside the HD image per slot (forward)
    uint32_t slot_cap;
    int32_t max_frames;
    AdjFrame* frames;
    uint32_t* counters;     // [0] pairs, [1] slots
    double* partials;       // per-block gradient partials (10 each)
    double* grad;           // 10 reduced gradient entries
};
// Camera of the HD image for the adjoint: K (fx, fy, cx, cy) and the
// depth-to-HD transform at the linearisation point.
struct AdjCamera {
    float fx, fy, cx, cy;
    float R[9], t[3];
    int32_t width, height, n_frames;
    int32_t nc[3];
    float s_c, origin[3];
};

// Device scratch for one frame.
struct Scratch {
    Counters* ctr;
    uint32_t* geo_list;
    uint32_t* vis_list;
    uint32_t* col_list;
    uint8_t* col_act;       // per geometry brick: active cells at its last band gate (capped at 255)
    uint32_t* depth_tiles;  // per 8x8 tile: min valid depth | max valid depth << 16
    float* depth_m;         // per pixel RN(D * 0.001) metres, -inf where D = 0
    uint8_t* bstate;        // per brick, this frame: bit 0 = in the geometry list, bit 1 = visible
    uint32_t* need;         // per visible brick: listed bricks among it and its + neighbours not yet updated
    unsigned long long* ready;  // ready queue of the fused frame: frame_tag << 32 | brick
    struct FuseSync* fsync;
    uint32_t* err;
    uint2* vox;           // colour voxels that passed the band gate this frame: x | y << 16, z
    uint32_t vox_cap;
};

// Per-axis tables of the colour grid, built once on the host with the band
// kernel's binary32 operations: for colour index k on axis a, the trilinear
// fraction of its centre (frac) and its geometry cell relative to the owning
// brick (cell, 0..7: the cell between brick voxels cell and cell + 1, voxel 8
// being the next brick's voxel 0); a brick owns the colour indices whose
// cell's lower corner lies in it.  For brick coordinate bb, the first owned
// colour index (k0[bb], owned range k0[bb] .. k0[bb + 1] - 1) and, per cell,
// the owned indices that fall in it (span[bb * 8 + cell] = first | end << 8,
// relative to k0[bb]); info[bb] = mask of the cells that own indices
// (8 bits) | most indices of one cell << 9.
struct AxisTables {
    const float* frac[3];
    const int8_t* cell[3];
    const int32_t* k0[3];
    const uint16_t* span[3];
    const uint16_t* info[3];
};

struct Volumes {
    float* F;
    uint8_t* W;
    uint32_t* C;
    BrickSummary* summ;
    AxisTables tab;
};

// ------------------------------------------------------------- launchers --
// All launchers queue work on `stream` and return cudaGetLastError().
cudaError_t launch_init_summaries(BrickSummary* summ, int64_t n, cudaStream_t stream);
// Queue the kernels of one frame.  `ev` (nullable) holds 7 events: ev[0] is
// recorded before the first kernel, then one after each of depth tiles, brick
// culling, geometry, colour list, colour band and colour voxels.
struct LaunchGrids {
    int geo, col, vox;  // persistent grid sizes (blocks) of the geometry and two colour kernels
    int fuse;           // persistent grid size of k_fused (every block resident)
};
// The same frame in two parts: depth tiles and brick culling (which read only
// the depth image, the brick summaries and the tile buffer) and the rest
// from the geometry update on.  `list_done` (nullable) is recorded after the
// colour list, the last reader of the brick lists and tiles of this frame.
// With c.fused the pre part also counts each visible brick's listed
// neighbours (k_need) and the post part runs k_fused (geometry, colour
// candidates and band gate in one launch) and then the colour voxels;
// `list_done` is then recorded after k_fused.
cudaError_t launch_frame_pre(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                             cudaStream_t stream, cudaEvent_t* ev);
cudaError_t launch_frame_post(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                              const uint8_t* rgb, const LaunchGrids& g, cudaStream_t stream, cudaEvent_t* ev,
                              cudaEvent_t list_done);
cudaError_t launch_frame(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                         const uint8_t* rgb, const LaunchGrids& g, cudaStream_t stream, cudaEvent_t* ev = nullptr);
int geometry_blocks_per_sm();
int geometry_linear_blocks_per_sm();  // k_geometry_linear (the allocation-free entry point)
int colour_blocks_per_sm();
int voxel_blocks_per_sm();
int fused_blocks_per_sm();

// Layout conversion between brick-major storage and linear x-fastest arrays,
// for z in [z0, z1).  `dst`/`src` point at the slab's first element.
cudaError_t launch_to_linear_f32(const float* brick, float* lin, const int32_t dims[3], int z0, int z1,
                                 cudaStream_t stream);
cudaError_t launch_to_linear_u8(const uint8_t* brick, uint8_t* lin, const int32_t dims[3], int z0, int z1,
                                cudaStream_t stream);
cudaError_t launch_to_linear_u32(const uint32_t* brick, uint32_t* lin, const int32_t dims[3], int z0, int z1,
                                 cudaStream_t stream);
cudaError_t launch_from_linear_f32(float* brick, const float* lin, const int32_t dims[3], int z0, int z1,
                                   cudaStream_t stream);
cudaError_t launch_from_linear_u8(uint8_t* brick, const uint8_t* lin, const int32_t dims[3], int z0, int z1,
                                  cudaStream_t stream);
cudaError_t launch_from_linear_u32(uint32_t* brick, const uint32_t* lin, const int32_t dims[3], int z0, int z1,
                                   cudaStream_t stream);
cudaError_t launch_recompute_summaries(const float* F, const uint8_t* W, BrickSummary* summ, const int32_t ng[3],
                                       float band, cudaStream_t stream);
constexpr float CELL_EPS = 1e-5f;  // bound on trilinear overshoot of the corner range

// Geometry-only fusion of one frame into caller-owned linear x-fastest F / w
// arrays, with caller-provided scratch (counters, depth tiles, brick list).
cudaError_t launch_geometry_static(const FrameConst& c, float* F, uint8_t* W, const uint16_t* depth, Counters* ctr,
                                   uint32_t* tiles, uint32_t* geo_list, int grid_geo, cudaStream_t stream);
// Frame constants of a volume description, by the same rules as tsdf_integrate.
struct VolumeDesc {
    int32_t ng[3];
    float s_g, origin[3], mu;
    int32_t max_weight;
};
void geometry_frame_constants(const VolumeDesc& d, const float Kd[9], const float Twd[16], int dw, int dh,
                              FrameConst& c);

// One scan of a batched frame step: its frame constants, volumes, scratch and
// this step's device images.
struct ScanDesc {
    FrameConst c;
    Volumes vol;
    Scratch scr;
    const uint16_t* depth;
    const uint8_t* rgb;
};
// Ready-queue counters of the fused frame (k_fused).
struct FuseSync {
    unsigned int head;   // queue entries taken
    unsigned int tail;   // queue entries pushed
    unsigned int stall;  // test injection: the next frame's count pass withholds one ready brick
    unsigned int claim;  // frame tag of the block that resets this frame's colour-side counters
    unsigned int open;   // frame tag once those counters are reset (colour work may start)
    unsigned int pad[3];
};
// Grid barrier and work counters of the batched persistent kernel.
struct BatchSync {
    unsigned int count;      // blocks arrived at the current barrier
    unsigned int gen;        // barrier generation
    unsigned int err;        // 1: a barrier wait gave up (bounded wait)
    unsigned int band_next;  // band-phase work counter
    unsigned int stall;      // test injection: block 0 skips the first barrier of the next step
    unsigned int pad[3];
};
constexpr int MAX_BATCH = 256;  // scans per batched launch
// One frame step of n scans in a single cooperative launch: depth tiles,
// bricks, geometry, colour candidates, band gate and colour voxels, with a
// bounded grid barrier between phases.  Scans are processed in descriptor
// order (put the largest first); the geometry and band phases hand out
// tiles of `tile` consecutive listed bricks of one scan per work item.
cudaError_t launch_batch_step(const ScanDesc* descs, int n, BatchSync* sync, int grid, int tile, cudaStream_t stream);
int batch_blocks_per_sm();
size_t batch_smem_bytes();

cudaError_t launch_frame_record(const FrameConst& c, const Volumes& v, const Scratch& s, const uint16_t* depth,
                                const LaunchGrids& g, const AdjBuffers& a, int frame, cudaStream_t stream);
cudaError_t launch_adjoint_finalize(const AdjBuffers& a, uint32_t n_pairs_max, cudaStream_t stream);
cudaError_t launch_adjoint_forward(const AdjCamera& cam, const AdjBuffers& a, uint32_t n_slots, const float* images,
                                   float* C, int32_t* n_out, cudaStream_t stream);
cudaError_t launch_adjoint_backward(const AdjCamera& cam, const AdjBuffers& a, uint32_t n_slots, const float* images,
                                    const float* grad_C, float* grad_images, int blocks, cudaStream_t stream);

// ------------------------------------------------------------ ray casting --
// Constants of one ray-casting call (see tsdf_raycast in tsdf.h): K^-1 and the
// camera pose (camera -> world), volume geometry, march range and steps.
struct RayConst {
    float Kinv[9], R[9], t[3];
    float origin[3];
    float s_g, inv_sg, inv_sc;
    float near_, far_, step_far, step_near;
    int32_t ng[3], nb[3], nc[3], ncb[3];
    int32_t width, height;
    uint32_t max_iter;  // bound on samples per ray (never reached for valid parameters)
};
cudaError_t launch_raycast(const RayConst& c, const float* F, const uint8_t* W, const uint32_t* C,
                           const BrickSummary* summ, float* range, float* vertex, float* normal, uint32_t* rgbw,
                           cudaStream_t stream);

// ------------------------------------------------------- camera tracking --
// One pyramid level of one tracking step (see tsdf_track in tsdf.h).
struct TrackLevel {
    int32_t w, h;
    float K[9];                    // level intrinsics (pinhole)
    const float *V, *N;            // current vertex / normal maps, camera frame, 3 floats per pixel
    const float *PV, *PN;          // predicted vertex / normal maps, world frame
    float Rp[9], tp[3];            // world -> camera of the prediction
    float max_dist2, min_cos;      // correspondence gates
};
// Depth pyramid in metres: d[l] of (W >> l) x (H >> l) floats.
cudaError_t launch_track_pyramid(const uint16_t* depth, int W, int H, int levels, float* const* d, cudaStream_t stream);
// Vertex and normal maps of one level; Kinv4 = (1/fx, 1/fy, -cx/fx, -cy/fy).
cudaError_t launch_track_maps(const float* d, int w, int h, const float Kinv4[4], float* V, float* N,
                              cudaStream_t stream);
int track_blocks(int npx);       // blocks (and binary64 partial-sum rows) of one step's reduction
size_t track_record_doubles();   // doubles recorded per step: 29 sums, 16 pose, 6 xi, 1 solved flag
// One Gauss-Newton step at the device pose (binary64 row-major 4x4, updated in place).
cudaError_t launch_track_step(const TrackLevel& L, double* pose, double* partials, double* record,
                              cudaStream_t stream);

// ------------------------------------------------- mesh and texture maps --
// Geometry of the volume for mesh extraction (see tsdf_mesh in tsdf.h).
struct MeshConst {
    int32_t ng[3], nb[3];
    float s_g;
    float origin[3];
};
// Candidate bricks (cells whose corners can have both signs), then one warp per
// candidate; triangles are appended at *count (slots beyond cap are counted,
// not written).
cudaError_t launch_mesh(const MeshConst& c, const float* F, const uint8_t* W, const BrickSummary* summ,
                        uint32_t* list, uint32_t* n_list, float* out, uint64_t cap, unsigned long long* count,
                        bool cubes, cudaStream_t stream);
// Copy the 256-entry marching-cubes case table (count, then edge triples) to
// the device.
cudaError_t upload_cube_cases(const uint8_t (*table)[16], cudaStream_t stream);
// Colour volume for texture maps (see tsdf_texture_fill in tsdf.h).
struct ColourConst {
    int32_t nc[3], ncb[3];
    float s_c, inv_sc;
    float origin[3];
};
// Eq. 11-12 sizes of n triangles into wh and their exclusive texel offsets
// into off[0..n] (block sums in `scratch`, (n + 1023) / 1024 + 1 entries).
cudaError_t launch_texture_layout(const float* tris, int64_t n, float size_pixel, int32_t max_side, int32_t* wh,
                                  int64_t* off, int64_t* scratch, cudaStream_t stream);
cudaError_t launch_texture_fill(const ColourConst& c, const uint32_t* C, const float* tris, int64_t n,
                                const int32_t* wh, const int64_t* off, int64_t total, uint32_t* texels,
                                cudaStream_t stream);

// ------------------------------------------------------------ addressing --
__host__ __device__ __forceinline__ int64_t brick_offset(int x, int y, int z, const int32_t nb[3]) {
    int64_t b = ((int64_t)(z >> 3) * nb[1] + (y >> 3)) * nb[0] + (x >> 3);
    return b * BRICK_VOX + (((z & 7) * BRICK + (y & 7)) * BRICK + (x & 7));
}

}  // namespace tsdf
