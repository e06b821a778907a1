// Host side of the batched C ABI (tsdf_batch_*): many independent scans, one
// frame each per step, fused by one persistent cooperative launch captured in
// a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"
#include "common.cuh"

using namespace tsdf;
using namespace tsdf_host;

struct tsdf_batch {
    std::vector<tsdf_volume*> vols;  // descriptor order: largest volume first
    std::vector<int> slot_of;        // caller index -> descriptor index
    cudaStream_t stream;
    int device;
    ScanDesc* d_descs[2];            // double-buffered descriptor tables
    ScanDesc* h_descs[2];            // page-locked host copies read by the graph's copy node
    cudaEvent_t copied[2];           // the step that last read h_descs[i] has copied it
    bool copied_valid[2];
    BatchSync* d_sync;
    int sms, max_blocks_per_sm, blocks_per_sm;
    int tile;  // listed bricks per work item of the geometry and band phases
    bool use_graph;
    cudaGraphExec_t exec[2];
    int step;
};

namespace {

void release_graphs(tsdf_batch* b) {
    for (auto& e : b->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

tsdf_status queue_step(tsdf_batch* b, int buf) {
    const int n = (int)b->vols.size();
    const size_t bytes = sizeof(ScanDesc) * n;
    const int grid = b->sms * b->blocks_per_sm;
    if (!b->use_graph) {
        cudaError_t e = cudaMemcpyAsync(b->d_descs[buf], b->h_descs[buf], bytes, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = launch_batch_step(b->d_descs[buf], n, b->d_sync, grid, b->tile, b->stream);
        return e == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
    }
    if (!b->exec[buf]) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return TSDF_ERR_CUDA;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_descs[buf], b->h_descs[buf], bytes, cudaMemcpyHostToDevice, cap);
        if (e == cudaSuccess) e = launch_batch_step(b->d_descs[buf], n, b->d_sync, grid, b->tile, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[buf], g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->exec[buf] = nullptr;
            return TSDF_ERR_CUDA;
        }
    }
    return cudaGraphLaunch(b->exec[buf], b->stream) == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

}  // namespace

extern "C" {

tsdf_status tsdf_batch_create(tsdf_volume* const* volumes, int32_t n, tsdf_batch** out) {
    if (!volumes || !out || n < 1 || n > MAX_BATCH) return TSDF_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!volumes[i]) return TSDF_ERR_INVALID_ARG;
        if (volumes[i]->stream != volumes[0]->stream || volumes[i]->device != volumes[0]->device)
            return fail(volumes[i], TSDF_ERR_INVALID_ARG, "batched volumes must share a device and a stream");
        if (volumes[i]->profiling) return fail(volumes[i], TSDF_ERR_INVALID_ARG, "disable profiling for batching");
        for (int j = 0; j < i; ++j)
            if (volumes[j] == volumes[i]) return TSDF_ERR_INVALID_ARG;
    }
    tsdf_batch* b = new (std::nothrow) tsdf_batch();
    if (!b) return TSDF_ERR_OOM;
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    auto work = [&](int i) {  // a scan's cost grows with its voxel count
        const tsdf_volume* v = volumes[i];
        return (double)v->ng[0] * v->ng[1] * v->ng[2] + (double)v->nc[0] * v->nc[1] * v->nc[2] / 4.0;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return work(a) > work(c); });
    b->slot_of.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        b->vols.push_back(volumes[idx[k]]);
        b->slot_of[idx[k]] = k;
    }
    b->stream = volumes[0]->stream;
    b->device = volumes[0]->device;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->max_blocks_per_sm = batch_blocks_per_sm();
    b->blocks_per_sm = b->max_blocks_per_sm;
    b->tile = 1;
    b->use_graph = true;
    tsdf_volume* v0 = volumes[0];
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) {
        b->d_descs[i] = (ScanDesc*)dev_alloc(v0, sizeof(ScanDesc) * n);
        ok = b->d_descs[i] && cudaHostAlloc((void**)&b->h_descs[i], sizeof(ScanDesc) * n, cudaHostAllocDefault) ==
                                  cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&b->copied[i], cudaEventDisableTiming) == cudaSuccess;
    }
    b->d_sync = ok ? (BatchSync*)dev_alloc(v0, sizeof(BatchSync)) : nullptr;
    if (!ok || !b->d_sync || cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream) != cudaSuccess) {
        cudaGetLastError();
        tsdf_batch_destroy(b);
        return TSDF_ERR_OOM;
    }
    *out = b;
    return TSDF_OK;
}

void tsdf_batch_destroy(tsdf_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    release_graphs(b);
    for (int i = 0; i < 2; ++i) {
        if (b->d_descs[i]) dev_free(b->vols[0], b->d_descs[i]);
        if (b->h_descs[i]) cudaFreeHost(b->h_descs[i]);
        if (b->copied[i]) cudaEventDestroy(b->copied[i]);
    }
    if (b->d_sync) dev_free(b->vols[0], b->d_sync);
    cudaGetLastError();
    delete b;
}

tsdf_status tsdf_batch_set_schedule(tsdf_batch* b, int32_t blocks_per_sm, int32_t bricks_per_item, int32_t use_graph) {
    if (!b || blocks_per_sm < 1 || blocks_per_sm > b->max_blocks_per_sm || bricks_per_item < 1 ||
        bricks_per_item > TSDF_BATCH_MAX_BRICKS_PER_ITEM)
        return TSDF_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    release_graphs(b);
    b->blocks_per_sm = blocks_per_sm;
    b->tile = bricks_per_item;
    b->use_graph = use_graph != 0;
    return TSDF_OK;
}

tsdf_status tsdf_batch_get_schedule(const tsdf_batch* b, int32_t* blocks_per_sm, int32_t* max_blocks_per_sm,
                                    int32_t* bricks_per_item, int32_t* use_graph) {
    if (!b) return TSDF_ERR_INVALID_ARG;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    if (max_blocks_per_sm) *max_blocks_per_sm = b->max_blocks_per_sm;
    if (bricks_per_item) *bricks_per_item = b->tile;
    if (use_graph) *use_graph = b->use_graph ? 1 : 0;
    return TSDF_OK;
}

tsdf_status tsdf_batch_integrate(tsdf_batch* b, const tsdf_frame* frames) {
    if (!b || !frames) return TSDF_ERR_INVALID_ARG;
    const int n = (int)b->vols.size();
    const int buf = b->step & 1;
    // the table is read by a copy queued two steps ago: wait for it
    if (b->copied_valid[buf] && cudaEventSynchronize(b->copied[buf]) != cudaSuccess) return TSDF_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        const tsdf_frame& f = frames[i];
        tsdf_volume* v = b->vols[b->slot_of[i]];
        if (!f.depth_mm || !f.rgb_hwc || !f.K_depth || !f.K_rgb || !f.T_world_depth || !f.T_depth_rgb)
            return fail(v, TSDF_ERR_INVALID_ARG, "NULL frame argument");
        if (f.dsz.width < 1 || f.dsz.height < 1 || f.csz.width < 1 || f.csz.height < 1 || f.dsz.width > 16384 ||
            f.dsz.height > 16384 || f.csz.width > 16384 || f.csz.height > 16384)
            return fail(v, TSDF_ERR_INVALID_ARG, "image size outside 1..16384");
        if (!is_device_ptr(f.depth_mm) || !is_device_ptr(f.rgb_hwc))
            return fail(v, TSDF_ERR_INVALID_ARG, "batched frames must be device images");
        float Ki[9];
        if (!finite_all(f.K_depth, 9) || !finite_all(f.K_rgb, 9) || !invert3(f.K_depth, Ki) || !invert3(f.K_rgb, Ki) ||
            !rigid_ok(f.T_world_depth) || !rigid_ok(f.T_depth_rgb) || !translation_ok(f.T_world_depth) ||
            !translation_ok(f.T_depth_rgb))
            return fail(v, TSDF_ERR_INVALID_ARG, "invalid intrinsics or transform");
        ScanDesc& d = b->h_descs[buf][b->slot_of[i]];
        frame_constants(v, f.K_depth, f.K_rgb, f.T_world_depth, f.T_depth_rgb, f.dsz.width, f.dsz.height,
                        f.csz.width, f.csz.height, d.c);
        const uint16_t* dd = nullptr;
        tsdf_status st = stage_depth(v, f.depth_mm, f.dsz, d.c.tiles_x * d.c.tiles_y, &dd);
        if (st != TSDF_OK) return st;
        d.vol = v->vol;
        d.scr = v->scr;
        d.depth = dd;
        d.rgb = f.rgb_hwc;
    }
    tsdf_status st = queue_step(b, buf);
    if (st != TSDF_OK) return fail(b->vols[0], st, "batched step launch");
    if (cudaEventRecord(b->copied[buf], b->stream) != cudaSuccess) return TSDF_ERR_CUDA;
    b->copied_valid[buf] = true;
    for (auto* v : b->vols) ++v->frames;
    ++b->step;
    return TSDF_OK;
}

tsdf_status tsdf_batch_synchronize(tsdf_batch* b) {
    if (!b) return TSDF_ERR_INVALID_ARG;
    BatchSync h;
    cudaError_t e = cudaMemcpyAsync(&h, b->d_sync, sizeof h, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(b->vols[0], e, "batch synchronize");
    if (h.err) {
        // clear the barrier state so the batch can be used again
        cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
        cudaStreamSynchronize(b->stream);
        return fail(b->vols[0], TSDF_ERR_TIMEOUT, "a grid barrier wait of the batched step gave up");
    }
    for (auto* v : b->vols) {
        tsdf_status s = check_device_error(v);
        if (s != TSDF_OK) return s;
    }
    return TSDF_OK;
}

tsdf_status tsdf_batch_inject_stall(tsdf_batch* b) {
    if (!b) return TSDF_ERR_INVALID_ARG;
    const unsigned one = 1u;
    cudaError_t e = cudaMemcpyAsync(&b->d_sync->stall, &one, sizeof one, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

// Native autotuner: times every schedule -- grid size (blocks per SM) times
// work-item size (1, 2, 4, 8 listed bricks per item) -- on clones of the
// batch's volumes with the given frames, interleaving the candidates over
// `rounds` rounds, and keeps the one with the smallest median step time.
tsdf_status tsdf_batch_autotune(tsdf_batch* b, const tsdf_frame* frames, int32_t rounds, int32_t* best_blocks_per_sm,
                                int32_t* best_bricks_per_item, float* ms_per_candidate) {
    if (!b || !frames || rounds < 1) return TSDF_ERR_INVALID_ARG;
    const int n = (int)b->vols.size();
    std::vector<tsdf_volume*> clones(n, nullptr);
    tsdf_status st = TSDF_OK;
    for (int i = 0; i < n && st == TSDF_OK; ++i) {  // clones in caller order
        const tsdf_volume* v = b->vols[b->slot_of[i]];
        tsdf_params p;
        tsdf_params_default(&p);
        for (int a = 0; a < 3; ++a) p.origin[a] = v->origin[a];
        p.sigma = v->sigma;
        p.band = v->band;
        p.colour_mode = v->colour_mode;
        p.sample_mode = v->sample_mode;
        p.culling = v->culling;
        p.update_free_space = v->free_space;
        p.stream = (void*)v->stream;
        p.allocator = v->alloc;
        st = tsdf_create_ex(v->ng, v->nc, v->s_g, v->mu, v->max_weight, &p, &clones[i]);
    }
    tsdf_batch* tb = nullptr;
    if (st == TSDF_OK) st = tsdf_batch_create(clones.data(), n, &tb);
    const int ntile = 4;  // 1, 2, 4, 8 bricks per item
    const int cands = b->max_blocks_per_sm * ntile;
    std::vector<std::vector<float>> times(cands);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == TSDF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = TSDF_ERR_CUDA;
    for (int r = 0; r < rounds && st == TSDF_OK; ++r)
        for (int k = 1; k <= cands && st == TSDF_OK; ++k) {
            st = tsdf_batch_set_schedule(tb, (k - 1) / ntile + 1, 1 << ((k - 1) % ntile), 0);
            if (st == TSDF_OK) st = tsdf_batch_integrate(tb, frames);  // warm the schedule
            if (st != TSDF_OK) break;
            cudaEventRecord(e0, tb->stream);
            st = tsdf_batch_integrate(tb, frames);
            cudaEventRecord(e1, tb->stream);
            if (st == TSDF_OK) st = tsdf_batch_synchronize(tb);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            times[k - 1].push_back(ms);
        }
    int best = (b->blocks_per_sm - 1) * ntile + 1;
    if (st == TSDF_OK) {
        float best_ms = 1e30f;
        for (int k = 1; k <= cands; ++k) {
            auto t = times[k - 1];
            std::sort(t.begin(), t.end());
            const float med = t.empty() ? 1e30f : t[t.size() / 2];
            if (ms_per_candidate) ms_per_candidate[k - 1] = med;
            if (med < best_ms) {
                best_ms = med;
                best = k;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    tsdf_batch_destroy(tb);
    for (auto* c : clones) tsdf_destroy(c);
    if (st != TSDF_OK) return st;
    const int bps = (best - 1) / ntile + 1, tile = 1 << ((best - 1) % ntile);
    if (best_blocks_per_sm) *best_blocks_per_sm = bps;
    if (best_bricks_per_item) *best_bricks_per_item = tile;
    return tsdf_batch_set_schedule(b, bps, tile, b->use_graph ? 1 : 0);
}

}  // extern "C"
