/*
 * tsdf.h — C ABI of the GB300 geometry-TSDF + asymmetric colour-volume fusion
 * library (libtsdf.so).
 *
 * The library fuses RGB-D frames into two volumes over the same cube:
 *   - a geometry volume: truncated signed distance F (binary32, normalised to
 *     [-1, 1] by the truncation distance mu) and an 8-bit weight w, the
 *     KinectFusion TSDF the paper builds on (Section III);
 *   - a colour volume with more voxels over the same extent (Section IV.B, the
 *     "asymmetric" colour volume), each voxel an 8-bit RGB colour C and an
 *     8-bit weight W packed as R | G<<8 | B<<16 | W<<24.
 * Each frame is a depth image (Kinect depth camera) and an HD RGB image from a
 * rigidly attached, calibrated camera (Section IV.A).
 *
 * Units and conventions
 *   - lengths in metres; depth images in uint16 millimetres, 0 = no measurement;
 *   - RGB images uint8, height x width x 3, R first, rows contiguous;
 *   - cameras: x right, y down, z forward; pixel (i, j) has its centre at
 *     image coordinates (i, j);
 *   - K: row-major 3x3 intrinsics (Eq. 1); T: row-major 4x4 rigid transforms;
 *   - T_world_depth maps depth-camera coordinates to world coordinates (the
 *     inverse of the motion (R_n, t_n) of Eq. 5); T_depth_rgb maps depth-camera
 *     coordinates to RGB-camera coordinates ([R_calib | t_calib], Eq. 3);
 *   - the volumes are axis-aligned in world coordinates; voxel (x, y, z) has
 *     its centre at origin + (index + 0.5) * voxel_size;
 *   - volumes returned by tsdf_read are linear, x fastest:
 *     index = (z * Ny + y) * Nx + x.
 *
 * Errors: every call returns a tsdf_status; no call aborts, throws across the
 * ABI or traps the device.  Kernel-side problems are recorded in a device
 * status word and reported by the next synchronising call (tsdf_read,
 * tsdf_synchronize, tsdf_save).
 *
 * Threading: one handle is used from one host thread at a time; work on a
 * handle is ordered on its CUDA stream.
 */
#ifndef TSDF_H
#define TSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsdf_volume tsdf_volume; /* opaque; owned by the library */

typedef enum {
    TSDF_OK = 0,
    TSDF_ERR_INVALID_ARG = -1,  /* an argument failed validation; nothing was done */
    TSDF_ERR_OOM = -2,          /* device memory could not be allocated */
    TSDF_ERR_CUDA = -3,         /* a CUDA runtime call failed (see tsdf_last_error) */
    TSDF_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up */
    TSDF_ERR_DEVICE_FAULT = -5, /* a kernel recorded an internal inconsistency */
    TSDF_ERR_IO = -6            /* checkpoint file could not be read or written */
} tsdf_status;

typedef struct {
    int32_t width, height;
} tsdf_image_size;

/* Device-memory provider.  alloc returns a device pointer (NULL on failure)
 * for `bytes` bytes, usable on `stream`; free releases it.  NULL alloc/free
 * select cudaMalloc/cudaFree.  The Python binding passes PyTorch's caching
 * allocator here. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} tsdf_allocator;

enum { TSDF_COLOUR_COUNT = 0, TSDF_COLOUR_PAPER_NORMAL = 1 };
enum { TSDF_SAMPLE_NEAREST = 0, TSDF_SAMPLE_BILINEAR = 1 };

/* Options of tsdf_create_ex.  Fill with tsdf_params_default first. */
typedef struct {
    float origin[3];           /* world position of the volumes' minimum corner;
                                  NaN = the cube centred on the world origin */
    float sigma;               /* depth-distance gate of Eq. 7, metres [0.020, the paper's 20 mm] */
    float band;                /* TSDF band gate on colour voxels, normalised units;
                                  NaN = one colour voxel: s_c / mu */
    int32_t colour_mode;       /* TSDF_COLOUR_COUNT: Eq. 9 with sample weight 1 (the
                                  weight counts observing frames, capped at max_weight);
                                  TSDF_COLOUR_PAPER_NORMAL: Eq. 8-10 */
    int32_t sample_mode;       /* TSDF_SAMPLE_NEAREST (the HD pixel of Eq. 9) or BILINEAR */
    int32_t culling;           /* 1: skip bricks that provably change nothing (results
                                  are identical either way); 0: sweep every brick */
    int32_t update_free_space; /* 1: voxels in front of the surface (sdf > mu) are
                                  updated with F = 1; 0: only |sdf| <= mu */
    void* stream;              /* cudaStream_t for all work on the handle; NULL = legacy default */
    tsdf_allocator allocator;
    int32_t slab_z[2];         /* {z0, z1}: the handle holds the z-slab [z0, z1) of the geometry
                                  volume dims_geo (and the same slice of space of the colour
                                  volume) instead of the whole volume; {0, 0} = whole [0, 0] */
} tsdf_params;

/* Fill *p with the defaults listed above. */
void tsdf_params_default(tsdf_params* p);

/* Create the two volumes, zero-initialised (F = 0, all weights 0).
 *   dims_geo    geometry voxels per axis (x, y, z), each 1..4096
 *   dims_col    colour voxels per axis; the same cube is split into more (or
 *               fewer) voxels: dims_col[i] * dims_geo[0] == dims_col[0] * dims_geo[i]
 *               and dims_col[i] <= 8 * dims_geo[i] (Section IV.B: same size,
 *               higher dimension; the paper uses a ratio of 2)
 *   voxel_size  geometry voxel edge s_g (m) > 0; the cube edge is dims_geo * s_g
 *               and the colour voxel edge s_c = dims_geo[0] * s_g / dims_col[0]
 *   mu          truncation distance (m) > 0
 *   max_weight  weight cap, 1..255 (weights count observing frames up to it)
 *   out         receives the handle (owned by the caller until tsdf_destroy)
 * Z-slabs (params->slab_z = {z0, z1}, 0 <= z0 < z1 <= dims_geo[2]): one scan's
 * volumes split along z over several handles (several GPUs, or a colour
 * volume larger than one device holds; Section IV.B notes that GPU memory
 * bounds the colour volume).  dims_geo / dims_col stay the whole volume's;
 * z0 * dims_col[2] and z1 * dims_col[2] must be multiples of dims_geo[2] (the
 * cuts fall on whole colour voxels).  The handle holds colour z
 * [z0 c, z1 c), c = dims_col[2] / dims_geo[2], and geometry z [max(0, z0 - 1),
 * min(dims_geo[2], z1 + 1)): one geometry voxel beyond the slab on each side,
 * integrated redundantly, which the trilinear band gate of the colour voxels
 * next to the cut reads.  Every voxel is computed at its global index, so
 * each slab's values equal the whole volume's bit for bit; every slab handle
 * receives every frame.  tsdf_read / tsdf_write / tsdf_save / tsdf_load
 * cover the held ranges (tsdf_get_info: held_geo_z, held_col_z); the
 * geometry of [z0, z1) and the colour of the colour range, concatenated over
 * the slabs in z order, are the whole volumes.  Ray casting, mesh extraction,
 * texture maps and the adjoint need a whole-volume handle.
 * The volumes must lie within 10^6 m of the world origin (|origin| +
 * dims * voxel size per axis).
 * Errors: INVALID_ARG (bad dims, ratio, sizes, slab or NULL out), OOM, CUDA. */
tsdf_status tsdf_create(const int32_t dims_geo[3], const int32_t dims_col[3], float voxel_size, float mu,
                        int32_t max_weight, tsdf_volume** out);
tsdf_status tsdf_create_ex(const int32_t dims_geo[3], const int32_t dims_col[3], float voxel_size, float mu,
                           int32_t max_weight, const tsdf_params* params, tsdf_volume** out);

/* Fuse one frame (Section IV.B): the geometry (TSDF) update of every geometry
 * voxel, then the colour update of every colour voxel against the updated
 * geometry:
 *   Eq. 5   voxel -> current depth camera with the inverse of T_world_depth
 *   Eq. 6   projection with K_depth; outside the image or D = 0 -> skipped
 *   TSDF    sdf = D/1000 - Z; sdf < -mu -> skipped; F <- (F w + min(1, sdf/mu)) / (w+1),
 *           w <- min(w+1, max_weight)
 *   Eq. 7   colour voxels farther than sigma from the back-projected depth pixel are skipped
 *   band    colour voxels whose trilinear TSDF has |F| > band are skipped
 *   Eq. 3-4 projection through T_depth_rgb and K_rgb into the HD image
 *   Eq. 9   C <- (C W + HD + floor((W+1)/2)) div (W+1) per channel, W <- min(W+1, max_weight)
 *           (colour_mode TSDF_COLOUR_PAPER_NORMAL: Eq. 8-10 instead)
 *   depth_mm  dsz.height x dsz.width uint16, host or device pointer
 *   rgb_hwc   csz.height x csz.width x 3 uint8, host or device pointer
 *   K_depth, K_rgb, T_world_depth, T_depth_rgb: host pointers, read before return
 * Host images are copied with cudaMemcpyAsync into one of two device staging
 * buffers, on an internal copy stream as soon as the frame before the
 * previous one has finished with that buffer (so the copy runs beside the
 * previous frame's geometry update), or, for the first frame after anything
 * that broke the frame sequence, on the volume's internal second stream
 * (which runs the frame's depth tiles and brick culling beside the previous
 * frame's colour kernels, and which the handle's stream waits for before the
 * frame's geometry update): pageable memory is consumed before the call
 * returns, page-locked memory by the time the handle's stream reaches the
 * frame's geometry update.  Device images are read in place by
 * kernels queued on the streams, after all work queued on the handle's
 * stream before the call (a device depth image then waits for the previous
 * frame's colour kernels too; see tsdf_set_device_inputs_ready).  In both
 * asynchronous cases the caller must not overwrite the buffer until the
 * handle's stream has passed the frame's last kernel.  The call is
 * asynchronous with respect to the host.
 * Errors: INVALID_ARG (NULL pointers, sizes outside 1..16384, non-finite or
 * singular K, non-finite or non-rigid T with |R^T R - I| > 1e-4, a
 * translation beyond 10^6 m), OOM, CUDA. */
tsdf_status tsdf_integrate(tsdf_volume* vol, const uint16_t* depth_mm, tsdf_image_size dsz, const uint8_t* rgb_hwc,
                           tsdf_image_size csz, const float K_depth[9], const float K_rgb[9],
                           const float T_world_depth[16], const float T_depth_rgb[16]);

/* How tsdf_integrate runs a frame (same results either way, bit for bit).
 *   TSDF_SCHEDULE_KERNELS  a chain of kernels: depth tiles, brick culling,
 *       geometry update, colour candidates, band gate, colour voxels.
 *   TSDF_SCHEDULE_FUSED    the geometry update, colour-candidate test and band
 *       gate in one persistent launch: the colour work of a visible brick
 *       starts as soon as the geometry of its 27-neighbourhood is updated
 *       (Section IV.B: the colour step reads the updated TSDF), beside the
 *       geometry of other bricks; then the colour voxels.  A pinhole K_depth
 *       is required (otherwise the frame runs as the kernel chain).  Its only
 *       waits are bounded (1 s); one that gives up makes the next
 *       synchronising call return TSDF_ERR_TIMEOUT (that frame's colour is
 *       then incomplete; its geometry is not) and the next frame starts clean.
 * The schedule applies from the next tsdf_integrate on.  Default: KERNELS.
 * Errors: INVALID_ARG (NULL handle, unknown schedule). */
enum { TSDF_SCHEDULE_KERNELS = 0, TSDF_SCHEDULE_FUSED = 1 };
tsdf_status tsdf_set_frame_schedule(tsdf_volume* vol, int32_t schedule);
tsdf_status tsdf_get_frame_schedule(const tsdf_volume* vol, int32_t* schedule);

/* ready = 1: the caller guarantees that the device images it passes to
 * tsdf_integrate are complete when the call is made (written before an
 * earlier tsdf_integrate call on this handle, or by work the caller has
 * synchronised with).  A device depth image is then read by the frame's
 * depth tiles and brick culling on the second stream as soon as the previous
 * frame's colour list is done, beside its band and colour kernels, instead
 * of after all work on the handle's stream.  Default 0.  Host images are
 * unaffected (they are copied at the call).
 * Errors: INVALID_ARG (NULL handle, ready not 0 or 1). */
tsdf_status tsdf_set_device_inputs_ready(tsdf_volume* vol, int32_t ready);

/* Test hook of the fused schedule's bounded waits: in the next fused frame
 * one visible brick is never released, so the wait for it runs out (no
 * fault, no trap); synchronous. */
tsdf_status tsdf_fused_inject_stall(tsdf_volume* vol);

/* Copy the volumes out, linear x-fastest (Section IV.B: each colour voxel
 * stores its fused RGB value and weight).  Each destination may be NULL (not
 * read) or a host or device pointer of dims_geo product floats (tsdf), bytes
 * (w_geo) or dims_col product uint32 (rgbw); for a z-slab handle, of the held
 * ranges (dims_geo[0] * dims_geo[1] * (held_geo_z[1] - held_geo_z[0]) and
 * likewise for colour).  Synchronous: returns after the copies are complete,
 * and reports any recorded device-side error. */
tsdf_status tsdf_read(tsdf_volume* vol, float* tsdf, uint8_t* w_geo, uint32_t* rgbw);

/* Overwrite the volumes from linear x-fastest arrays (host or device), e.g. to
 * resume from a previous state.  Any argument may be NULL (left unchanged). */
tsdf_status tsdf_write(tsdf_volume* vol, const float* tsdf, const uint8_t* w_geo, const uint32_t* rgbw);

/* Wait for all queued work on the handle and report recorded device errors. */
tsdf_status tsdf_synchronize(tsdf_volume* vol);

/* Checkpoint: a little-endian file holding a header (magic "TSDFVOL1",
 * version, dims, voxel size, mu, max_weight, origin, sigma, band, modes, frame
 * count) then F, w and the packed colours, linear x-fastest.  tsdf_load needs
 * a handle created with the same dims; it restores the arrays and the frame
 * count.  Errors: IO, INVALID_ARG (header mismatch). */
tsdf_status tsdf_save(tsdf_volume* vol, const char* path);
tsdf_status tsdf_load(tsdf_volume* vol, const char* path);

/* Release the volumes and the handle.  NULL is ignored. */
void tsdf_destroy(tsdf_volume* vol);

/* Change the stream used by later calls on the handle. */
tsdf_status tsdf_set_stream(tsdf_volume* vol, void* stream);

/* Read-only description of a handle. */
typedef struct {
    int32_t dims_geo[3], dims_col[3];
    float voxel_geo, voxel_col;  /* s_g, s_c (m) */
    float origin[3];
    float mu, sigma, band;
    int32_t max_weight, colour_mode, sample_mode, culling, update_free_space;
    int64_t frames;              /* frames integrated so far */
    int64_t device_bytes;        /* bytes of device memory the handle holds */
    int32_t slab_z[2];           /* the slab [z0, z1) of a z-slab handle; {0, dims_geo[2]} otherwise */
    int32_t held_geo_z[2];       /* geometry z range held (the slab and its one-voxel margins) */
    int32_t held_col_z[2];       /* colour z range held */
} tsdf_info;
tsdf_status tsdf_get_info(const tsdf_volume* vol, tsdf_info* out);

/* Work counters (read synchronously).  The first group covers the most
 * recent tsdf_integrate: voxels whose geometry / colour was updated, and the
 * bricks (8^3 geometry voxels) the geometry and colour kernels processed.
 * The totals cover every frame since creation or the last
 * tsdf_profile_enable. */
typedef struct {
    int64_t geo_updated, col_updated;
    int64_t geo_bricks, col_bricks, visible_bricks, total_bricks;
    int64_t frames_counted;
    int64_t total_geo_updated, total_col_updated, total_geo_bricks, total_col_bricks, total_visible_bricks;
    /* totals of: colour candidate bricks holding at least one trilinear cell
     * that can pass the band gate, such cells, and geometry bricks in which
     * at least one voxel was updated */
    int64_t total_col_active_bricks, total_cells, total_geo_changed_bricks;
} tsdf_stats;
tsdf_status tsdf_get_stats(tsdf_volume* vol, tsdf_stats* out);

/* Asynchronous form of tsdf_get_stats, for a caller that queues frame k + 1
 * before it reads frame k's counters.  tsdf_stats_request queues, after the
 * work queued so far, a copy of the counters (TSDF_STATS_COPY_BYTES bytes,
 * device to page-locked host memory owned by the volume) into slot 0 or 1,
 * and returns without waiting.  After a frame integrated with its depth tiles
 * and culling on the volume's second stream it queues two such copies: one on
 * the second stream once the frame's colour list is done (for the counters
 * the next frame's depth tiles reset, which it precedes) and one on the
 * volume's stream (for the rest); after any other frame one copy on the
 * volume's stream, which the next frame's depth tiles then wait for.
 * tsdf_stats_collect waits for that slot's last request and fills *out as
 * tsdf_get_stats would have at the time of the request (a slot never
 * requested reads as zeros).  Slots other than 0 and 1 and NULL pointers are
 * rejected with TSDF_ERR_INVALID_ARG. */
#define TSDF_STATS_COPY_BYTES 128
tsdf_status tsdf_stats_request(tsdf_volume* vol, int32_t slot);
tsdf_status tsdf_stats_collect(tsdf_volume* vol, int32_t slot, tsdf_stats* out);

/* Phase timing.  While enabled, tsdf_integrate records CUDA events on the
 * handle's stream around each phase of a frame; tsdf_profile_read waits for
 * them and returns the accumulated device time per phase (milliseconds) and
 * the number of frames timed.  Enabling resets the accumulators and the
 * stats totals.  Timing adds event records between kernels and nothing else. */
enum {
    TSDF_PHASE_UPLOAD = 0,      /* host -> device copies of the frame */
    TSDF_PHASE_DEPTH_TILES = 1, /* per-tile depth range */
    TSDF_PHASE_BRICKS = 2,      /* brick culling and work lists */
    TSDF_PHASE_GEOMETRY = 3,    /* TSDF update */
    TSDF_PHASE_COLOUR_LIST = 4, /* colour candidate list */
    TSDF_PHASE_COLOUR_CELLS = 5, /* active trilinear cells of the candidates */
    TSDF_PHASE_COLOUR = 6,      /* colour update of the cells' colour voxels */
    TSDF_PHASE_COUNT = 7
};
typedef struct {
    int64_t frames;
    double ms[TSDF_PHASE_COUNT];
} tsdf_profile_report;
tsdf_status tsdf_profile_enable(tsdf_volume* vol, int32_t enable);
tsdf_status tsdf_profile_read(tsdf_volume* vol, tsdf_profile_report* out);
/* Restrict timing to the phases in mask (bit k = phase k; default all):
 * events are recorded only at the boundaries of those phases, so a single
 * timed kernel costs two event records per frame instead of eight.  Phases
 * outside the mask report 0 ms.  Errors: INVALID_ARG (mask outside
 * 1 .. 2^TSDF_PHASE_COUNT - 1). */
tsdf_status tsdf_profile_phases(tsdf_volume* vol, uint32_t mask);

/* ------------------------------------------------------------------------
 * Batched fusion: many independent scans (volumes of any sizes), one frame
 * each per step, fused by one persistent cooperative kernel launch, captured
 * in a CUDA graph, whose phases (depth tiles, bricks, geometry, colour
 * candidates, band gate, colour voxels) each span all scans, separated by a
 * grid barrier whose waits are bounded (1 s).  Results are identical to
 * calling tsdf_integrate on each volume.
 * ---------------------------------------------------------------------- */
typedef struct tsdf_batch tsdf_batch;

/* One scan's frame; fields as in tsdf_integrate.  Images must be device
 * pointers, valid until the step has run. */
typedef struct {
    const uint16_t* depth_mm;
    tsdf_image_size dsz;
    const uint8_t* rgb_hwc;
    tsdf_image_size csz;
    const float* K_depth;       /* 9, host */
    const float* K_rgb;         /* 9, host */
    const float* T_world_depth; /* 16, host */
    const float* T_depth_rgb;   /* 16, host */
} tsdf_frame;

/* A batch over n (1..256) distinct volumes sharing one device and stream
 * (the batch keeps them in descending size order internally).  The volumes
 * stay owned by the caller and must outlive the batch. */
tsdf_status tsdf_batch_create(tsdf_volume* const* volumes, int32_t n, tsdf_batch** out);
/* Fuse frames[i] into volume i (the caller's order) for every scan; queued
 * on the volumes' stream. */
tsdf_status tsdf_batch_integrate(tsdf_batch* batch, const tsdf_frame* frames);
/* Wait for queued steps; TSDF_ERR_TIMEOUT if a grid-barrier wait gave up
 * (the barrier state is then reset; that step's scans are left partially
 * updated), or a volume's recorded device error. */
tsdf_status tsdf_batch_synchronize(tsdf_batch* batch);
/* Schedule: blocks per SM of the persistent launch (1..max, the occupancy
 * limit) and whether steps replay a CUDA graph. */
/* The schedule of the batched step: blocks per SM of the persistent grid
 * (1..max_blocks_per_sm), listed bricks per work item of the geometry and
 * band phases (1..TSDF_BATCH_MAX_BRICKS_PER_ITEM: a warp takes that many
 * consecutive bricks of one scan's list at a time) and whether the step runs
 * as a CUDA graph.  Results do not depend on the schedule. */
#define TSDF_BATCH_MAX_BRICKS_PER_ITEM 8
tsdf_status tsdf_batch_set_schedule(tsdf_batch* batch, int32_t blocks_per_sm, int32_t bricks_per_item,
                                    int32_t use_graph);
tsdf_status tsdf_batch_get_schedule(const tsdf_batch* batch, int32_t* blocks_per_sm, int32_t* max_blocks_per_sm,
                                    int32_t* bricks_per_item, int32_t* use_graph);
/* Autotuner: times every schedule (blocks per SM 1..max_blocks_per_sm times
 * 1, 2, 4 or 8 bricks per item; median over `rounds` interleaved rounds) on
 * freshly created clones of the batch's volumes fed with `frames`, keeps the
 * fastest in the batch's schedule and reports it; ms_per_candidate
 * (nullable) receives 4 * max_blocks_per_sm median times, candidate
 * (blocks - 1) * 4 + log2(bricks per item).  The batch's own volumes are not
 * touched. */
tsdf_status tsdf_batch_autotune(tsdf_batch* batch, const tsdf_frame* frames, int32_t rounds,
                                int32_t* best_blocks_per_sm, int32_t* best_bricks_per_item, float* ms_per_candidate);
/* Failure injection for tests: in the next step one block never arrives at
 * the first grid barrier, so the other blocks' bounded waits run out. */
tsdf_status tsdf_batch_inject_stall(tsdf_batch* batch);
void tsdf_batch_destroy(tsdf_batch* batch);

/* ------------------------------------------------------------------------
 * Photometric colour loss and its adjoint (calibration refinement of the HD
 * camera).  Not in the paper, which takes the calibration of Section IV.A as
 * given: this differentiates the fused colour volume with respect to the HD
 * images, the HD intrinsics (Eq. 4) and the depth-to-HD extrinsic (Eq. 3).
 *
 * Over a recorded frame sequence, S_k is the set of colour voxels that pass
 * the depth-side gates of frame k (Eq. 5, Eq. 6 frustum and D > 0, Eq. 7 and
 * the trilinear band gate, against the geometry after frame k's update); it
 * does not depend on the HD camera.  For each voxel v in the union of the S_k
 * the forward pass gives the unrounded mean of its bilinear HD samples over
 * the frames whose 2x2 sample footprint lies inside the image,
 *   C_v = (1/n_v) sum_k bilinear(I_k, K_hd T P_vc)   (Eq. 9 with W = 1),
 * and the backward pass maps dL/dC to dL/dI_k, dL/dK_hd = (fx, fy, cx, cy)
 * and dL/dxi for a left perturbation T(xi) = exp(xi^) T of the extrinsic at
 * the given T, xi = (rho, phi), translation first.
 * ---------------------------------------------------------------------- */
typedef struct tsdf_adjoint tsdf_adjoint;

/* Buffers for up to max_frames (1..64) recorded frames and max_pairs
 * (frame, voxel) pairs, drawn from vol's allocator; vol provides the geometry
 * volume, its stream and scratch.  Errors: INVALID_ARG, OOM. */
tsdf_status tsdf_adjoint_create(tsdf_volume* vol, int32_t max_frames, int64_t max_pairs, tsdf_adjoint** out);
/* Fuse the geometry of one frame into vol (as tsdf_integrate does) and record
 * S_k; arguments as in tsdf_integrate.  Frames are numbered 0.. in order. */
tsdf_status tsdf_adjoint_record(tsdf_adjoint* adj, const uint16_t* depth_mm, tsdf_image_size dsz,
                                const float K_depth[9], const float T_world_depth[16]);
/* Close the recording: builds the voxel union (n_voxels slots).  Errors: OOM
 * when a buffer overflowed during recording. */
tsdf_status tsdf_adjoint_finalize(tsdf_adjoint* adj, int64_t* n_voxels);
/* Linear colour index of each slot (n_voxels uint32, host or device). */
tsdf_status tsdf_adjoint_voxels(tsdf_adjoint* adj, uint32_t* voxels);
/* The recorded (voxel, frame) pairs, grouped by frame in recording order and
 * in no fixed order within a frame (uint32 linear colour index, uint8 frame;
 * host or device; either may be NULL), and their count. */
tsdf_status tsdf_adjoint_pairs(tsdf_adjoint* adj, uint32_t* voxels, uint8_t* frames, int64_t* n_pairs);
/* Forward pass.  images: device float32 n_frames x csz.height x csz.width x 3
 * HD intensities; K_rgb4 = (fx, fy, cx, cy); T_depth_rgb row-major 4x4 (host).
 * colours: device float32 n_voxels x 3; counts: device int32 n_voxels (n_v).
 * Asynchronous on vol's stream. */
tsdf_status tsdf_adjoint_forward(tsdf_adjoint* adj, const float* images, tsdf_image_size csz, const float K_rgb4[4],
                                 const float T_depth_rgb[16], float* colours, int32_t* counts);
/* Backward pass at the camera of the preceding forward pass.  grad_colours:
 * device float32 n_voxels x 3 (dL/dC); grad_images: device float32 like
 * images, ACCUMULATED into; grad_theta: host double[10] = dL/d(fx, fy, cx, cy,
 * rho, phi).  Synchronous (returns after grad_theta is written). */
tsdf_status tsdf_adjoint_backward(tsdf_adjoint* adj, const float* images, tsdf_image_size csz, const float K_rgb4[4],
                                  const float T_depth_rgb[16], const float* grad_colours, float* grad_images,
                                  double grad_theta[10]);
void tsdf_adjoint_destroy(tsdf_adjoint* adj);

/* Allocation-free geometry fusion.  (The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory, for example code
 * running while another framework owns the device allocator, or a host with a
 * device-memory budget fixed in advance.)
 *
 * Fuses one depth frame into a caller-owned TSDF volume with the same
 * arithmetic and the same results as the geometry step of tsdf_integrate
 * (culling only skips bricks that cannot change).  It needs no handle and
 * calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (work counters, depth tiles, brick work list) is one fixed device array of
 * TSDF_STATIC_SCRATCH_BYTES = 256 + 4 * TSDF_STATIC_MAX_DEPTH_TILES +
 * 4 * TSDF_STATIC_MAX_BRICKS = 5,243,136 bytes (5.0 MiB) that every GPU
 * loading the library holds until the process exits.
 *   dims            voxels per axis (x, y, z), 1..4096, with at most
 *                   TSDF_STATIC_MAX_BRICKS bricks of 8^3 voxels
 *   voxel_size, mu, max_weight, origin   as in tsdf_create_ex
 *   tsdf_dev, w_dev device (or managed) arrays of dims[0]*dims[1]*dims[2] floats / bytes,
 *                   linear x-fastest, read and updated in place (start from
 *                   zeros for an empty volume)
 *   depth_dev       device uint16 millimetre depth image of dsz, at most
 *                   TSDF_STATIC_MAX_DEPTH_TILES tiles of 8x8 pixels
 *   K_depth, T_world_depth  host pointers, as in tsdf_integrate
 *   stream          cudaStream_t the kernels are queued on (NULL = legacy default)
 * Sizes beyond the maxima, NULL or host pointers and invalid K / T are
 * rejected with TSDF_ERR_INVALID_ARG before any work is queued.  The first
 * call on a device looks up the scratch array's device address there
 * (cudaGetSymbolAddress), so make it before any stream capture; the address
 * is kept for the life of the process, so do not use the library across a
 * cudaDeviceReset.  Every call shares the one scratch
 * array, which keeps the previous call's contents (the call clears what must
 * start at zero): calls whose work overlaps on the GPU race, so queue them on
 * one stream or wait between them.  Asynchronous with respect to the host. */
#define TSDF_STATIC_MAX_BRICKS (1 << 20)     /* e.g. 512^3 voxels use 262,144 bricks */
#define TSDF_STATIC_MAX_DEPTH_TILES 262144   /* e.g. 4096 x 4096 pixels use 262,144 tiles */
#define TSDF_STATIC_SCRATCH_BYTES (256 + 4 * TSDF_STATIC_MAX_DEPTH_TILES + 4 * TSDF_STATIC_MAX_BRICKS)
tsdf_status tsdf_integrate_geometry_static(const int32_t dims[3], float voxel_size, float mu, int32_t max_weight,
                                           const float origin[3], float* tsdf_dev, uint8_t* w_dev,
                                           const uint16_t* depth_dev, tsdf_image_size dsz, const float K_depth[9],
                                           const float T_world_depth[16], void* stream);

/* ------------------------------------------------------------------------
 * Camera tracking (Section III: the KinectFusion loop the paper builds on).
 * A vertex map and normal map pyramid is computed from the input depth map
 * and the camera motion is estimated by iterative closest point against the
 * surface vertex map predicted by ray tracing the geometry volume.  The paper
 * gives no more detail; the steps (all binary32 per pixel, in this order):
 *   pyramid   level 0: d = D * 0.001 m (D = 0: none); level l + 1 pixel (x, y):
 *             the mean of the valid depths of level l's block (2x + i, 2y + j),
 *             taken (0,0), (1,0), (0,1), (1,1), that lie within 0.03 m of the
 *             block's first valid depth (summed in that order, divided once);
 *             level l is W >> l by H >> l with f_l = f / 2^l and
 *             c_l = (c + 1/2) / 2^l - 1/2 (binary64, rounded once)
 *   maps      V = d (fmaf(1/fx, x, -cx/fx), fmaf(1/fy, y, -cy/fy), 1) (the
 *             coefficients binary64, rounded once); N = n / sqrt(n . n) with
 *             n = (V(x, y+1) - V) x (V(x+1, y) - V), facing the camera; no
 *             normal on the last row / column or next to a pixel without depth
 *   predict   per level, tsdf_raycast from T_world_depth_prev with the level's
 *             intrinsics and size (vertex and normal maps, world frame)
 *   steps     levels coarsest first, iterations[l] Gauss-Newton steps each:
 *             for a pixel with a vertex and a normal, p = R V + t, m = R N
 *             (R, t: the current pose rounded to binary32); the prediction
 *             pixel of q_c = R_p p + t_p (R_p = R_prev^T, t_p = -R_prev^T t_prev
 *             in binary64 rounded once) projected as in Eq. 6 (u = fmaf(fx, X,
 *             cx Z) * (1/Z), nearest, inside, Z > 0) with a predicted normal nq
 *             and vertex q; |p - q|^2 <= max_distance^2 and m . nq >=
 *             min_normal_cos; r = (p - q) . nq, J = (nq, p x nq).  A = sum J J^T,
 *             g = sum J r in binary64; xi = -A^-1 g by Cholesky (binary64; a
 *             matrix that is not positive definite leaves the pose), applied
 *             as T <- exp(xi^) T with xi = (rho, phi) (Rodrigues, binary64).
 * The pose stays on the device between steps: a frame's steps are queued
 * without host round trips.
 * ---------------------------------------------------------------------- */
#define TSDF_TRACK_MAX_LEVELS 3
#define TSDF_TRACK_MAX_STEPS 32
typedef struct {
    int32_t levels;                             /* 1..3 [3] */
    int32_t iterations[TSDF_TRACK_MAX_LEVELS];  /* steps per level, finest first [10, 5, 4]; total <= 32 */
    float max_distance;                         /* correspondence gate, metres [0.1] */
    float min_normal_cos;                       /* normal gate, cosine of the largest angle [cos 20 deg] */
    float near_m, far_m;                        /* prediction ray-cast range [0.1, 4] */
} tsdf_track_params;
void tsdf_track_params_default(tsdf_track_params* p);

/* What each step saw: its level, correspondences, sum of squared residuals,
 * the normal equations (A row-major, g), the pose it started from and whether
 * it was solved. */
typedef struct {
    int32_t steps;
    int32_t level[TSDF_TRACK_MAX_STEPS];
    int32_t solved[TSDF_TRACK_MAX_STEPS];
    int64_t correspondences[TSDF_TRACK_MAX_STEPS];
    double err2[TSDF_TRACK_MAX_STEPS];
    double A[TSDF_TRACK_MAX_STEPS][36];
    double g[TSDF_TRACK_MAX_STEPS][6];
    double T_before[TSDF_TRACK_MAX_STEPS][16];
} tsdf_track_report;

/* Track one depth frame against the volume (whole-volume handles only).
 *   depth_mm            dsz.height x dsz.width uint16 mm, host or device
 *   K_depth             pinhole 3x3 (zero skew, bottom row 0 0 1), host
 *   T_world_depth_prev  the pose the prediction is ray-cast from (row-major 4x4, host)
 *   T_init              the first estimate of the frame's pose (binary64, host)
 *   params              NULL = defaults
 *   T_out               the estimate after the last step (binary64, host)
 *   report              nullable
 * Synchronous.  Errors: INVALID_ARG (sizes, K, T, params, slab handle), OOM,
 * CUDA. */
tsdf_status tsdf_track(tsdf_volume* vol, const uint16_t* depth_mm, tsdf_image_size dsz, const float K_depth[9],
                       const float T_world_depth_prev[16], const double T_init[16], const tsdf_track_params* params,
                       double T_out[16], tsdf_track_report* report);

/* ------------------------------------------------------------------------
 * Ray casting of the fused volumes.  The paper shows the scan to the user by
 * ray casting the geometry and colour volumes (abstract) and tracks the camera
 * against a surface vertex map predicted by ray tracing the geometry volume
 * (Section III).  Output goes to plain buffers (no graphics API).
 *
 * Per pixel (x, y) of a camera with intrinsics K and pose T_world_camera
 * (camera -> world, x right, y down, z forward), all binary32:
 *   dc = K^-1 (x, y, 1) (K^-1 in binary64 rounded once), d = R dc / |dc|,
 *   p(t) = o + t d per axis as fmaf(t, d, o), t the distance from the camera
 *   centre o.  The TSDF at p is the trilinear interpolation used by the colour
 *   band gate (it exists only when its 8 corners are inside the volume and
 *   observed).  From t = near, samples step by step_near where the TSDF exists
 *   and is < 1 (inside the truncation band) and by step_far elsewhere; the first
 *   sample with TSDF <= 0 whose previous sample had TSDF > 0 is a hit, refined
 *   by linear interpolation of the zero crossing; the march ends without a hit
 *   once t > far.  At the hit vertex v: the normal is the normalised central
 *   difference of the TSDF over +-1 geometry voxel along each axis (pointing to
 *   free space; (0, 0, 0) when a difference sample does not exist) and the
 *   colour is the packed RGBW of the colour voxel holding v (0 outside).
 * ---------------------------------------------------------------------- */
typedef struct {
    float near_m, far_m;    /* march range along each ray, metres: 0 <= near < far <= 1000 */
    float step_far;         /* step outside the truncation band, metres; 0 = mu / 2 */
    float step_near;        /* step inside it, metres; 0 = geometry voxel / 2; needs far / step_near <= 2^22 */
} tsdf_raycast_params;

/* Ray-cast width x height pixels.  Outputs (any may be NULL; host or device
 * pointers, row-major, pixel (x, y) at y * width + x): range (float, the hit's
 * t, 0 for a miss), vertex and normal (3 floats per pixel, world frame, zero
 * for a miss), rgbw (packed colour, 0 for a miss or outside the colour
 * volume).  Ordered on the volume's stream; returns after host outputs are
 * written, device outputs are ready when the stream reaches that point.
 * Errors: INVALID_ARG (NULL vol or K/T, size outside 1..16384, non-finite or
 * singular K, T not a rigid motion, bad range or steps), OOM. */
tsdf_status tsdf_raycast(tsdf_volume* vol, const float K[9], const float T_world_camera[16], tsdf_image_size size,
                         const tsdf_raycast_params* params, float* range, float* vertex, float* normal,
                         uint32_t* rgbw);

/* ------------------------------------------------------------------------
 * Mesh extraction and per-polygon texture maps.  The paper extracts a polygon
 * mesh from the TSDF volume (Section IV.C) and textures each polygon with its
 * own 2D map sampled from the colour volume (Section IV.D, Eq. 11-14).
 *
 * Mesh: the zero level set of the TSDF by marching cubes (Section IV.C).  A
 * cell is the cube of eight neighbouring geometry voxels (corner k = (k & 1,
 * (k >> 1) & 1, k >> 2)) and is meshed only when all eight are observed; a
 * corner is inside when F < 0.  The twelve cell edges are numbered 4 a + r
 * (a the edge's axis, r the rank of its lower corner among the four corners
 * whose bit a is 0).  On each face, corners taken counter-clockwise about the
 * outward normal, every maximal run c_i..c_j of inside corners is cut off by
 * a segment from the edge (c_(i-1), c_i) to the edge (c_j, c_(j+1)), so a face
 * with two diagonal inside corners separates them.  The segments form closed
 * loops, taken in the order of their lowest edge; each loop is fanned along
 * the segments' direction from its first vertex (in loop order from the
 * lowest edge) whose fan has no triangle with all three vertices on one face
 * (else from the lowest edge), which winds every triangle with its normal to
 * free space (F > 0).  At most five triangles per cell; the library builds
 * its 256-case table from these rules.  The vertex on edge (p, q), p the lower
 * voxel index: t = F_p / (F_p - F_q), v = fmaf(t, P_q - P_p, P_p), P the voxel
 * centre fmaf(i + 1/2, s_g, origin).  Binary32, operation order as written.
 *
 * Marching tetrahedra (tsdf_mesh_ex, TSDF_MESH_TETRAHEDRA): each observed cell
 * is split into six tetrahedra along the diagonal from corner 0 to corner 7
 * (for each axis order (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x):
 * corners 0, 0 + a0, 0 + a0 + a1, 7), the same split on both sides of a shared
 * face.  A tetrahedron with a lone corner gives the triangle on its three
 * edges; one with two inside corners i1, i2 and outside corners o1, o2
 * (tetrahedron order) gives the quad on edges (i1,o1), (i1,o2), (i2,o2),
 * (i2,o1) as triangles ((i1,o1), (i1,o2), (i2,o2)) and ((i1,o1), (i2,o2),
 * (i2,o1)), wound so that their normal points to free space.
 * ---------------------------------------------------------------------- */
/* Write up to capacity triangles (9 floats each: v0, v1, v2; host or device
 * pointer, may be NULL with capacity 0) in no fixed order and set
 * *n_triangles to the number the volume has (more than capacity means the
 * output was cut short: call again with more room).  Errors: INVALID_ARG,
 * OOM. */
tsdf_status tsdf_mesh(tsdf_volume* vol, float* triangles, int64_t capacity, int64_t* n_triangles);
/* The same with a choice of method: TSDF_MESH_CUBES (what tsdf_mesh does) or
 * TSDF_MESH_TETRAHEDRA. */
enum { TSDF_MESH_CUBES = 0, TSDF_MESH_TETRAHEDRA = 1 };
tsdf_status tsdf_mesh_ex(tsdf_volume* vol, int32_t method, float* triangles, int64_t capacity, int64_t* n_triangles);

/* Texture map layout (Eq. 11-12): for n triangles (V_a, V_b, V_c as 9 floats
 * each) and the size of a texel on the model, w = max(2, round(|V_a V_b| /
 * size_pixel)) and h = max(2, round(|V_a V_c| / size_pixel)) (round half up,
 * at most max_side), written to wh (2n int32: w, h), and the texel offsets of
 * the maps laid one after another (offsets: n + 1 int64, offsets[n] = total).
 * Pointers host or device.  Errors: INVALID_ARG, OOM. */
tsdf_status tsdf_texture_layout(tsdf_volume* vol, const float* triangles, int64_t n, float size_pixel,
                                int32_t max_side, int32_t* wh, int64_t* offsets);
/* Texture maps (Eq. 13-14): texel (i, j) of triangle t, i the column along
 * V_aV_green = V_aV_b / (w - 1) and j the row along V_aV_blue = V_aV_c / (h - 1),
 * lies at V_a + i V_aV_green + j V_aV_blue and takes the trilinear
 * interpolation of the colour volume there over observed colour voxels only
 * (each channel rounded half up; alpha 255; 0 when no corner is observed).
 * Maps are row-major (h rows of w texels) at texels + offsets[t], packed
 * R | G << 8 | B << 16 | A << 24.  wh and offsets as tsdf_texture_layout gave
 * them; pointers host or device.  Errors: INVALID_ARG, OOM. */
tsdf_status tsdf_texture_fill(tsdf_volume* vol, const float* triangles, int64_t n, const int32_t* wh,
                              const int64_t* offsets, uint32_t* texels);

/* Human-readable text of a status, and the last error message of a handle
 * (empty if none).  The strings are owned by the library. */
const char* tsdf_status_string(tsdf_status s);
const char* tsdf_last_error(const tsdf_volume* vol);

#ifdef __cplusplus
}
#endif
#endif /* TSDF_H */
