// C ABI of camera tracking (tsdf_track in tsdf.h): validation, buffers, the
// per-level prediction ray casts and the queue of Gauss-Newton steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace tsdf_host;

namespace {

// Temporary device buffers of one call, freed when it returns.
struct Scratchpad {
    tsdf_volume* v;
    std::vector<void*> ptrs;
    explicit Scratchpad(tsdf_volume* vol) : v(vol) {}
    template <typename T>
    T* get(size_t n) {
        void* p = dev_alloc(v, n * sizeof(T) + 16);
        if (p) ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratchpad() {
        cudaStreamSynchronize(v->stream);
        for (void* p : ptrs) dev_free(v, p);
    }
};

bool pinhole_K(const float K[9]) {
    return finite_all(K, 9) && K[1] == 0.0f && K[3] == 0.0f && K[6] == 0.0f && K[7] == 0.0f && K[8] == 1.0f &&
           K[0] > 0.0f && K[4] > 0.0f;
}

}  // namespace

extern "C" void tsdf_track_params_default(tsdf_track_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->levels = 3;
    p->iterations[0] = 10;
    p->iterations[1] = 5;
    p->iterations[2] = 4;
    p->max_distance = 0.1f;
    p->min_normal_cos = (float)std::cos(20.0 * 3.14159265358979323846 / 180.0);
    p->near_m = 0.1f;
    p->far_m = 4.0f;
}

extern "C" tsdf_status tsdf_track(tsdf_volume* v, const uint16_t* depth_mm, tsdf_image_size dsz, const float K_depth[9],
                                  const float T_world_depth_prev[16], const double T_init[16],
                                  const tsdf_track_params* params, double T_out[16], tsdf_track_report* report) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (v->zoff_g != 0 || v->ng[2] != v->ngz_all) return fail(v, TSDF_ERR_INVALID_ARG, "track: needs a whole volume");
    if (!depth_mm || !K_depth || !T_world_depth_prev || !T_init || !T_out)
        return fail(v, TSDF_ERR_INVALID_ARG, "track: NULL argument");
    tsdf_track_params p;
    tsdf_track_params_default(&p);
    if (params) p = *params;
    int total = 0;
    if (p.levels < 1 || p.levels > TSDF_TRACK_MAX_LEVELS) return fail(v, TSDF_ERR_INVALID_ARG, "track: levels 1..3");
    for (int l = 0; l < p.levels; ++l) {
        if (p.iterations[l] < 0) return fail(v, TSDF_ERR_INVALID_ARG, "track: negative iteration count");
        total += p.iterations[l];
    }
    if (total > TSDF_TRACK_MAX_STEPS) return fail(v, TSDF_ERR_INVALID_ARG, "track: more than 32 steps");
    if ((dsz.width >> (p.levels - 1)) < 2 || (dsz.height >> (p.levels - 1)) < 2 || dsz.width > 16384 ||
        dsz.height > 16384)
        return fail(v, TSDF_ERR_INVALID_ARG, "track: image too small for the pyramid or larger than 16384");
    if (!pinhole_K(K_depth)) return fail(v, TSDF_ERR_INVALID_ARG, "track: K must be a finite pinhole matrix");
    if (!rigid_ok(T_world_depth_prev)) return fail(v, TSDF_ERR_INVALID_ARG, "track: T_world_depth_prev not rigid");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_init[i])) return fail(v, TSDF_ERR_INVALID_ARG, "track: T_init not finite");
    if (!(p.max_distance > 0.0f) || !std::isfinite(p.max_distance) || !(p.min_normal_cos >= -1.0f) ||
        !(p.min_normal_cos <= 1.0f))
        return fail(v, TSDF_ERR_INVALID_ARG, "track: bad gates");

    Scratchpad sp(v);
    const int W = dsz.width, H = dsz.height;
    cudaError_t e = cudaSuccess;
    const uint16_t* d_depth = depth_mm;
    if (!is_device_ptr(depth_mm)) {
        uint16_t* buf = sp.get<uint16_t>((size_t)W * H);
        if (!buf) return fail(v, TSDF_ERR_OOM, "track: depth staging");
        e = cudaMemcpyAsync(buf, depth_mm, (size_t)W * H * sizeof(uint16_t), cudaMemcpyHostToDevice, v->stream);
        d_depth = buf;
    }
    float* dl[TSDF_TRACK_MAX_LEVELS];
    float *Vl[TSDF_TRACK_MAX_LEVELS], *Nl[TSDF_TRACK_MAX_LEVELS], *PVl[TSDF_TRACK_MAX_LEVELS],
        *PNl[TSDF_TRACK_MAX_LEVELS];
    for (int l = 0; l < p.levels; ++l) {
        const size_t n = (size_t)(W >> l) * (H >> l);
        dl[l] = sp.get<float>(n);
        Vl[l] = sp.get<float>(3 * n);
        Nl[l] = sp.get<float>(3 * n);
        PVl[l] = sp.get<float>(3 * n);
        PNl[l] = sp.get<float>(3 * n);
        if (!dl[l] || !Vl[l] || !Nl[l] || !PVl[l] || !PNl[l]) return fail(v, TSDF_ERR_OOM, "track: level buffers");
    }
    const size_t rec_n = tsdf::track_record_doubles();
    double* pose = sp.get<double>(16);
    double* partials = sp.get<double>((size_t)tsdf::track_blocks(W * H) * 29);
    double* records = sp.get<double>((size_t)TSDF_TRACK_MAX_STEPS * rec_n);
    if (!pose || !partials || !records) return fail(v, TSDF_ERR_OOM, "track: step buffers");
    if (e == cudaSuccess) e = cudaMemcpyAsync(pose, T_init, 16 * sizeof(double), cudaMemcpyHostToDevice, v->stream);
    if (e == cudaSuccess) e = tsdf::launch_track_pyramid(d_depth, W, H, p.levels, dl, v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "track: pyramid");

    // world -> prediction camera, as the fusion's frame constants invert a pose
    tsdf::TrackLevel L;
    std::memset(&L, 0, sizeof L);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) L.Rp[r * 3 + k] = T_world_depth_prev[k * 4 + r];
    for (int i = 0; i < 3; ++i) {
        double s = (double)T_world_depth_prev[0 * 4 + i] * (double)T_world_depth_prev[0 * 4 + 3];
        s = s + (double)T_world_depth_prev[1 * 4 + i] * (double)T_world_depth_prev[1 * 4 + 3];
        s = s + (double)T_world_depth_prev[2 * 4 + i] * (double)T_world_depth_prev[2 * 4 + 3];
        L.tp[i] = (float)(-s);
    }
    L.max_dist2 = p.max_distance * p.max_distance;
    L.min_cos = p.min_normal_cos;
    tsdf_raycast_params rp = {p.near_m, p.far_m, 0.0f, 0.0f};
    int step = 0;
    int step_level[TSDF_TRACK_MAX_STEPS];
    for (int l = p.levels - 1; l >= 0; --l) {
        const int w = W >> l, h = H >> l;
        const double s = std::ldexp(1.0, -l);
        float Kl[9] = {0.0f};
        Kl[0] = (float)((double)K_depth[0] * s);
        Kl[4] = (float)((double)K_depth[4] * s);
        Kl[2] = (float)(((double)K_depth[2] + 0.5) * s - 0.5);
        Kl[5] = (float)(((double)K_depth[5] + 0.5) * s - 0.5);
        Kl[8] = 1.0f;
        const float kinv4[4] = {(float)(1.0 / (double)Kl[0]), (float)(1.0 / (double)Kl[4]),
                                (float)(-(double)Kl[2] / (double)Kl[0]), (float)(-(double)Kl[5] / (double)Kl[4])};
        e = tsdf::launch_track_maps(dl[l], w, h, kinv4, Vl[l], Nl[l], v->stream);
        if (e != cudaSuccess) return cuda_fail(v, e, "track: maps");
        tsdf::RayConst rc;
        const tsdf_status rs = raycast_constants(v, Kl, T_world_depth_prev, tsdf_image_size{w, h}, &rp, rc);
        if (rs != TSDF_OK) return rs;
        e = tsdf::launch_raycast(rc, v->vol.F, v->vol.W, v->vol.C, v->vol.summ, nullptr, PVl[l], PNl[l], nullptr,
                                 v->stream);
        if (e != cudaSuccess) return cuda_fail(v, e, "track: prediction");
        L.w = w;
        L.h = h;
        std::memcpy(L.K, Kl, sizeof Kl);
        L.V = Vl[l];
        L.N = Nl[l];
        L.PV = PVl[l];
        L.PN = PNl[l];
        for (int it = 0; it < p.iterations[l]; ++it, ++step) {
            step_level[step] = l;
            e = tsdf::launch_track_step(L, pose, partials, records + (size_t)step * rec_n, v->stream);
            if (e != cudaSuccess) return cuda_fail(v, e, "track: step");
        }
    }
    std::vector<double> rec((size_t)std::max(step, 1) * rec_n);
    e = cudaMemcpyAsync(T_out, pose, 16 * sizeof(double), cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess && step)
        e = cudaMemcpyAsync(rec.data(), records, (size_t)step * rec_n * sizeof(double), cudaMemcpyDeviceToHost,
                            v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "track: read-back");
    if (report) {
        std::memset(report, 0, sizeof *report);
        report->steps = step;
        for (int k = 0; k < step; ++k) {
            const double* r = rec.data() + (size_t)k * rec_n;
            int q = 0;
            for (int a = 0; a < 6; ++a)
                for (int b = a; b < 6; ++b, ++q) report->A[k][a * 6 + b] = report->A[k][b * 6 + a] = r[q];
            for (int a = 0; a < 6; ++a) report->g[k][a] = r[21 + a];
            report->err2[k] = r[27];
            report->correspondences[k] = (int64_t)r[28];
            for (int i = 0; i < 16; ++i) report->T_before[k][i] = r[29 + i];
            report->solved[k] = r[29 + 16 + 6] != 0.0;
            report->level[k] = step_level[k];
        }
    }
    return TSDF_OK;
}
