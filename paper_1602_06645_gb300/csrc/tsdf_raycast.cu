// C ABI of the ray caster (tsdf_raycast in tsdf.h): validation, constants,
// launch, and the copy to host outputs.
#include <cmath>
#include <cstring>

#include "api_internal.h"

using namespace tsdf_host;

namespace {

// Device buffer for one output: the caller's pointer when it is device
// memory, else a temporary that is copied to the host afterwards.
struct Out {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool staged = false;
};

tsdf_status prepare(tsdf_volume* v, void* user, size_t bytes, Out& o) {
    o.user = user;
    o.bytes = bytes;
    if (!user) return TSDF_OK;
    if (is_device_ptr(user)) {
        o.dev = user;
        return TSDF_OK;
    }
    o.dev = dev_alloc(v, bytes);
    o.staged = true;
    return o.dev ? TSDF_OK : fail(v, TSDF_ERR_OOM, "ray-cast output staging buffer");
}

}  // namespace

namespace tsdf_host {
tsdf_status raycast_constants(tsdf_volume* v, const float K[9], const float T_world_camera[16], tsdf_image_size size,
                              const tsdf_raycast_params* params, tsdf::RayConst& c) {
    if (size.width < 1 || size.height < 1 || size.width > 16384 || size.height > 16384)
        return fail(v, TSDF_ERR_INVALID_ARG, "raycast: image size outside 1..16384");
    if (!finite_all(K, 9) || !finite_all(T_world_camera, 16) || !rigid_ok(T_world_camera))
        return fail(v, TSDF_ERR_INVALID_ARG, "raycast: K must be finite and T_world_camera a rigid motion");
    std::memset(&c, 0, sizeof c);
    if (!invert3(K, c.Kinv)) return fail(v, TSDF_ERR_INVALID_ARG, "raycast: K is singular");
    tsdf_raycast_params p = params ? *params : tsdf_raycast_params{0.1f, 4.0f, 0.0f, 0.0f};
    if (p.step_far == 0.0f) p.step_far = (float)(0.5 * (double)v->mu);
    if (p.step_near == 0.0f) p.step_near = (float)(0.5 * (double)v->s_g);
    if (!(p.near_m >= 0.0f) || !(p.far_m > p.near_m) || !(p.far_m <= 1000.0f) || !(p.step_near > 0.0f) ||
        !(p.step_far >= p.step_near) || !((double)p.far_m / (double)p.step_near <= 4194304.0) ||
        !std::isfinite(p.step_far))
        return fail(v, TSDF_ERR_INVALID_ARG, "raycast: need 0 <= near < far <= 1000, 0 < step_near <= step_far, "
                                             "far / step_near <= 2^22");
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.R[r * 3 + k] = T_world_camera[r * 4 + k];
        c.t[r] = T_world_camera[r * 4 + 3];
        c.origin[r] = v->origin[r];
        c.ng[r] = v->ng[r];
        c.nb[r] = v->nb[r];
        c.nc[r] = v->nc[r];
        c.ncb[r] = v->ncb[r];
    }
    c.s_g = v->s_g;
    c.inv_sg = (float)(1.0 / (double)v->s_g);
    c.inv_sc = (float)(1.0 / (double)v->s_c);
    c.near_ = p.near_m;
    c.far_ = p.far_m;
    c.step_far = p.step_far;
    c.step_near = p.step_near;
    c.width = size.width;
    c.height = size.height;
    // each step adds at least step_near less its rounding; 2% and 16 samples of slack
    c.max_iter = (uint32_t)std::ceil(1.02 * ((double)p.far_m - (double)p.near_m) / (double)p.step_near) + 16u;
    return TSDF_OK;
}
}  // namespace tsdf_host

extern "C" tsdf_status tsdf_raycast(tsdf_volume* v, const float K[9], const float T_world_camera[16],
                                    tsdf_image_size size, const tsdf_raycast_params* params, float* range,
                                    float* vertex, float* normal, uint32_t* rgbw) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (v->zoff_g != 0 || v->ng[2] != v->ngz_all) return fail(v, TSDF_ERR_INVALID_ARG, "raycast: needs a whole volume");
    if (!K || !T_world_camera) return fail(v, TSDF_ERR_INVALID_ARG, "raycast: K and T_world_camera are required");
    tsdf::RayConst c;
    const tsdf_status cs = raycast_constants(v, K, T_world_camera, size, params, c);
    if (cs != TSDF_OK) return cs;

    const size_t npx = (size_t)size.width * size.height;
    Out o_range, o_vertex, o_normal, o_rgbw;
    tsdf_status st = prepare(v, range, npx * sizeof(float), o_range);
    if (st == TSDF_OK) st = prepare(v, vertex, 3 * npx * sizeof(float), o_vertex);
    if (st == TSDF_OK) st = prepare(v, normal, 3 * npx * sizeof(float), o_normal);
    if (st == TSDF_OK) st = prepare(v, rgbw, npx * sizeof(uint32_t), o_rgbw);
    bool staged = false;
    if (st == TSDF_OK) {
        cudaError_t e = tsdf::launch_raycast(c, v->vol.F, v->vol.W, v->vol.C, v->vol.summ, (float*)o_range.dev,
                                             (float*)o_vertex.dev, (float*)o_normal.dev, (uint32_t*)o_rgbw.dev,
                                             v->stream);
        for (Out* o : {&o_range, &o_vertex, &o_normal, &o_rgbw}) {
            if (e != cudaSuccess || !o->staged) continue;
            e = cudaMemcpyAsync(o->user, o->dev, o->bytes, cudaMemcpyDeviceToHost, v->stream);
            staged = true;
        }
        if (e == cudaSuccess && staged) e = cudaStreamSynchronize(v->stream);
        if (e != cudaSuccess) st = cuda_fail(v, e, "raycast");
    }
    if (staged || st != TSDF_OK) cudaStreamSynchronize(v->stream);
    for (Out* o : {&o_range, &o_vertex, &o_normal, &o_rgbw})
        if (o->staged && o->dev) dev_free(v, o->dev);
    return st;
}
