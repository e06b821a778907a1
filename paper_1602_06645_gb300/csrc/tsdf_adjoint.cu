// Host side of the adjoint C ABI (tsdf_adjoint_*): gate recording over a
// frame sequence, then forward (fused colours) and backward (gradients with
// respect to the HD images, K_hd and the se(3) extrinsic) passes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"
#include "common.cuh"

using namespace tsdf;
using namespace tsdf_host;

struct tsdf_adjoint {
    tsdf_volume* vol;
    int32_t max_frames;
    int64_t pair_cap, slot_cap;
    int32_t n_frames;
    bool finalized;
    uint32_t n_slots;
    std::vector<AdjFrame> frames;
    AdjBuffers buf;
    int grad_blocks;
    void* allocs[16];
    int n_allocs;
};

namespace {

void* adj_alloc(tsdf_adjoint* a, size_t bytes) {
    void* p = dev_alloc(a->vol, bytes);
    if (p) a->allocs[a->n_allocs++] = p;
    return p;
}

AdjCamera camera(const tsdf_adjoint* a, const float K4[4], const float T[16], tsdf_image_size csz) {
    AdjCamera c;
    std::memset(&c, 0, sizeof c);
    c.fx = K4[0];
    c.fy = K4[1];
    c.cx = K4[2];
    c.cy = K4[3];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.R[r * 3 + k] = T[r * 4 + k];
        c.t[r] = T[r * 4 + 3];
    }
    c.width = csz.width;
    c.height = csz.height;
    c.n_frames = a->n_frames;
    tsdf_info info;
    tsdf_get_info(a->vol, &info);
    for (int i = 0; i < 3; ++i) {
        c.nc[i] = info.dims_col[i];
        c.origin[i] = info.origin[i];
    }
    c.s_c = info.voxel_col;
    return c;
}

bool camera_ok(const float K4[4], const float T[16], tsdf_image_size csz) {
    return K4 && T && finite_all(K4, 4) && K4[0] != 0.0f && K4[1] != 0.0f && rigid_ok(T) && csz.width >= 2 &&
           csz.height >= 2 && csz.width <= 16384 && csz.height <= 16384;
}

}  // namespace

extern "C" {

tsdf_status tsdf_adjoint_create(tsdf_volume* vol, int32_t max_frames, int64_t max_pairs, tsdf_adjoint** out) {
    if (!vol || !out || max_frames < 1 || max_frames > 64 || max_pairs < 1 || max_pairs > (int64_t(1) << 31))
        return TSDF_ERR_INVALID_ARG;
    if (vol->zoff_g != 0 || vol->ng[2] != vol->ngz_all) return TSDF_ERR_INVALID_ARG;  // whole volumes only
    *out = nullptr;
    tsdf_info info;
    tsdf_get_info(vol, &info);
    const int64_t ncv = (int64_t)info.dims_col[0] * info.dims_col[1] * info.dims_col[2];
    if (ncv > (int64_t)0x7FFFFFFF) return fail(vol, TSDF_ERR_INVALID_ARG, "colour volume too large for the adjoint");
    tsdf_adjoint* a = new (std::nothrow) tsdf_adjoint();
    if (!a) return TSDF_ERR_OOM;
    a->vol = vol;
    a->max_frames = max_frames;
    a->pair_cap = max_pairs;
    a->slot_cap = std::min<int64_t>(max_pairs, ncv);
    AdjBuffers& b = a->buf;
    b.pair_cap = (uint32_t)a->pair_cap;
    b.slot_cap = (uint32_t)a->slot_cap;
    b.max_frames = max_frames;
    b.pair_vox = (uint32_t*)adj_alloc(a, (size_t)a->pair_cap * 4);
    b.pair_frame = (uint8_t*)adj_alloc(a, (size_t)a->pair_cap);
    b.slot_of = (int32_t*)adj_alloc(a, (size_t)ncv * 4);
    b.V = (uint32_t*)adj_alloc(a, (size_t)a->slot_cap * 4);
    b.slot_count = (uint32_t*)adj_alloc(a, (size_t)a->slot_cap * 4);
    b.slot_frames = (uint8_t*)adj_alloc(a, (size_t)a->slot_cap * max_frames);
    b.n_valid = (int32_t*)adj_alloc(a, (size_t)a->slot_cap * 4);
    b.frames = (AdjFrame*)adj_alloc(a, sizeof(AdjFrame) * max_frames);
    b.counters = (uint32_t*)adj_alloc(a, 64);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, vol->device);
    a->grad_blocks = std::max(1, sms * 4);
    b.partials = (double*)adj_alloc(a, sizeof(double) * 10 * a->grad_blocks);
    b.grad = (double*)adj_alloc(a, sizeof(double) * 10);
    if (a->n_allocs != 11) {  // adj_alloc keeps only the allocations that succeeded
        tsdf_adjoint_destroy(a);
        return fail(vol, TSDF_ERR_OOM, "adjoint buffers");
    }
    if (cudaMemsetAsync(b.counters, 0, 64, vol->stream) != cudaSuccess) {
        tsdf_adjoint_destroy(a);
        return TSDF_ERR_CUDA;
    }
    *out = a;
    return TSDF_OK;
}

void tsdf_adjoint_destroy(tsdf_adjoint* a) {
    if (!a) return;
    cudaStreamSynchronize(a->vol->stream);
    for (int i = 0; i < a->n_allocs; ++i) dev_free(a->vol, a->allocs[i]);
    delete a;
}

tsdf_status tsdf_adjoint_record(tsdf_adjoint* a, const uint16_t* depth_mm, tsdf_image_size dsz, const float K_depth[9],
                                const float T_world_depth[16]) {
    if (!a) return TSDF_ERR_INVALID_ARG;
    tsdf_volume* v = a->vol;
    if (a->finalized) return fail(v, TSDF_ERR_INVALID_ARG, "adjoint already finalized");
    if (a->n_frames >= a->max_frames) return fail(v, TSDF_ERR_INVALID_ARG, "more frames than reserved");
    if (!depth_mm || !K_depth || !T_world_depth) return fail(v, TSDF_ERR_INVALID_ARG, "NULL argument");
    if (dsz.width < 1 || dsz.height < 1 || dsz.width > 16384 || dsz.height > 16384)
        return fail(v, TSDF_ERR_INVALID_ARG, "image size outside 1..16384");
    float Kdi[9];
    if (!finite_all(K_depth, 9) || !invert3(K_depth, Kdi) || !rigid_ok(T_world_depth))
        return fail(v, TSDF_ERR_INVALID_ARG, "invalid intrinsics or pose");
    const float I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    FrameConst c;
    frame_constants(v, K_depth, K_depth, T_world_depth, I, dsz.width, dsz.height, dsz.width, dsz.height, c);
    c.record_mode = 1;
    const uint16_t* d_depth = nullptr;
    tsdf_status st = stage_depth(v, depth_mm, dsz, c.tiles_x * c.tiles_y, &d_depth);
    if (st != TSDF_OK) return st;
    cudaError_t e = launch_frame_record(c, v->vol, v->scr, d_depth, v->grids, a->buf, a->n_frames, v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "adjoint record launch");
    AdjFrame f;
    std::memcpy(f.R, c.R, sizeof f.R);
    std::memcpy(f.t, c.t, sizeof f.t);
    a->frames.push_back(f);
    ++a->n_frames;
    ++v->frames;
    return TSDF_OK;
}

tsdf_status tsdf_adjoint_finalize(tsdf_adjoint* a, int64_t* n_voxels) {
    if (!a) return TSDF_ERR_INVALID_ARG;
    tsdf_volume* v = a->vol;
    cudaStream_t s = v->stream;
    AdjBuffers& b = a->buf;
    tsdf_info info;
    tsdf_get_info(v, &info);
    const size_t ncv = (size_t)info.dims_col[0] * info.dims_col[1] * info.dims_col[2];
    uint32_t host_ctr[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(b.frames, a->frames.data(), sizeof(AdjFrame) * a->frames.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.slot_of, 0xFF, ncv * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.slot_count, 0, (size_t)a->slot_cap * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.counters + 1, 0, 8, s);
    if (e == cudaSuccess) e = launch_adjoint_finalize(b, (uint32_t)a->pair_cap, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_ctr, b.counters, sizeof host_ctr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(v, e, "adjoint finalize");
    tsdf_status st = check_device_error(v);
    if (st != TSDF_OK) return fail(v, TSDF_ERR_OOM, "gate recording overflowed its buffers");
    if (host_ctr[0] > b.pair_cap || host_ctr[2]) return fail(v, TSDF_ERR_OOM, "adjoint pair/slot buffers too small");
    a->n_slots = std::min<uint32_t>(host_ctr[1], b.slot_cap);
    a->finalized = true;
    if (n_voxels) *n_voxels = a->n_slots;
    return TSDF_OK;
}

tsdf_status tsdf_adjoint_voxels(tsdf_adjoint* a, uint32_t* voxels) {
    if (!a || !voxels || !a->finalized) return TSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(voxels, a->buf.V, (size_t)a->n_slots * 4, cudaMemcpyDefault, a->vol->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->vol->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(a->vol, e, "adjoint voxels");
}

tsdf_status tsdf_adjoint_pairs(tsdf_adjoint* a, uint32_t* voxels, uint8_t* frames, int64_t* n_pairs) {
    if (!a || !n_pairs) return TSDF_ERR_INVALID_ARG;
    uint32_t n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, a->buf.counters, 4, cudaMemcpyDeviceToHost, a->vol->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->vol->stream);
    if (e != cudaSuccess) return cuda_fail(a->vol, e, "adjoint pairs");
    n = std::min<uint32_t>(n, a->buf.pair_cap);
    if (voxels) e = cudaMemcpyAsync(voxels, a->buf.pair_vox, (size_t)n * 4, cudaMemcpyDefault, a->vol->stream);
    if (e == cudaSuccess && frames) e = cudaMemcpyAsync(frames, a->buf.pair_frame, n, cudaMemcpyDefault, a->vol->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->vol->stream);
    *n_pairs = n;
    return e == cudaSuccess ? TSDF_OK : cuda_fail(a->vol, e, "adjoint pairs");
}

tsdf_status tsdf_adjoint_forward(tsdf_adjoint* a, const float* images, tsdf_image_size csz, const float K_rgb4[4],
                                 const float T_depth_rgb[16], float* colours, int32_t* counts) {
    if (!a || !images || !colours || !counts) return TSDF_ERR_INVALID_ARG;
    if (!a->finalized) return fail(a->vol, TSDF_ERR_INVALID_ARG, "adjoint not finalized");
    if (!camera_ok(K_rgb4, T_depth_rgb, csz)) return fail(a->vol, TSDF_ERR_INVALID_ARG, "invalid HD camera");
    AdjCamera cam = camera(a, K_rgb4, T_depth_rgb, csz);
    cudaError_t e = launch_adjoint_forward(cam, a->buf, a->n_slots, images, colours, counts, a->vol->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(a->vol, e, "adjoint forward");
}

tsdf_status tsdf_adjoint_backward(tsdf_adjoint* a, const float* images, tsdf_image_size csz, const float K_rgb4[4],
                                  const float T_depth_rgb[16], const float* grad_colours, float* grad_images,
                                  double grad_theta[10]) {
    if (!a || !images || !grad_colours || !grad_images || !grad_theta) return TSDF_ERR_INVALID_ARG;
    if (!a->finalized) return fail(a->vol, TSDF_ERR_INVALID_ARG, "adjoint not finalized");
    if (!camera_ok(K_rgb4, T_depth_rgb, csz)) return fail(a->vol, TSDF_ERR_INVALID_ARG, "invalid HD camera");
    AdjCamera cam = camera(a, K_rgb4, T_depth_rgb, csz);
    cudaError_t e = launch_adjoint_backward(cam, a->buf, a->n_slots, images, grad_colours, grad_images, a->grad_blocks,
                                            a->vol->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad_theta, a->buf.grad, sizeof(double) * 10, cudaMemcpyDeviceToHost, a->vol->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->vol->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(a->vol, e, "adjoint backward");
}

}  // extern "C"
