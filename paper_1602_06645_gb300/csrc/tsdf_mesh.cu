// C ABI of mesh extraction and texture maps (tsdf_mesh, tsdf_texture_layout,
// tsdf_texture_fill in tsdf.h): validation, staging of host buffers, launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace tsdf_host;

namespace {

// Temporary device buffers of one call, freed when it returns.
struct Temps {
    tsdf_volume* v;
    std::vector<void*> ptrs;
    explicit Temps(tsdf_volume* vol) : v(vol) {}
    void* get(size_t bytes) {
        void* p = dev_alloc(v, bytes ? bytes : 16);
        if (p) ptrs.push_back(p);
        return p;
    }
    ~Temps() {
        if (!ptrs.empty()) cudaStreamSynchronize(v->stream);
        for (void* p : ptrs) dev_free(v, p);
    }
};

// Device view of an input: the pointer itself when it is device memory, else
// a temporary copy.
const void* input(tsdf_volume* v, Temps& t, const void* p, size_t bytes, cudaError_t& e) {
    if (!p || is_device_ptr(p)) return p;
    void* d = t.get(bytes);
    if (!d) return nullptr;
    if (bytes) e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, v->stream);
    return d;
}

// Device buffer for an output (the pointer itself, or a temporary that
// finish() copies back).
void* output(Temps& t, void* p, size_t bytes) { return (!p || is_device_ptr(p)) ? p : t.get(bytes); }

cudaError_t finish(tsdf_volume* v, void* user, const void* dev, size_t bytes) {
    if (!user || user == dev || !bytes) return cudaSuccess;
    return cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, v->stream);
}

tsdf::MeshConst mesh_const(const tsdf_volume* v) {
    tsdf::MeshConst c;
    std::memset(&c, 0, sizeof c);
    for (int a = 0; a < 3; ++a) {
        c.ng[a] = v->ng[a];
        c.nb[a] = v->nb[a];
        c.origin[a] = v->origin[a];
    }
    c.s_g = v->s_g;
    return c;
}

// ---------------------------------------------------- marching-cubes cases --
// The 256-case table of tsdf.h's marching-cubes rules, built once.  Corner k
// sits at (k & 1, (k >> 1) & 1, k >> 2); edge 4 a + r joins the r-th corner
// with bit a clear (in increasing order) to its neighbour along a.
struct CubeCases {
    uint8_t t[256][16];  // triangle count, then edge triples
};

int cube_edge(int p, int q) {
    const int lo = std::min(p, q), a = (p ^ q) == 1 ? 0 : ((p ^ q) == 2 ? 1 : 2);
    // drop bit a of the lower corner: its rank among the corners with bit a clear
    return 4 * a + (((lo >> (a + 1)) << a) | (lo & ((1 << a) - 1)));
}

// The four corners of the face (axis a, side s) counter-clockwise about its
// outward normal: with u = a + 1, v = a + 2 (mod 3) the frame (a, u, v) is
// right-handed, so about +a the turn runs u -> v and about -a it runs v -> u.
void face_ring(int a, int s, int ring[4]) {
    const int u = (a + 1) % 3, v = (a + 2) % 3;
    const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    for (int i = 0; i < 4; ++i) {
        const int iu = s ? uv[i][0] : uv[i][1], iv = s ? uv[i][1] : uv[i][0];
        ring[i] = (s << a) | (iu << u) | (iv << v);
    }
}

bool edges_share_a_face(const int e[3]) {
    for (int b = 0; b < 3; ++b)
        for (int side = 0; side < 2; ++side) {
            bool all = true;
            for (int k = 0; k < 3; ++k) {
                const int a = e[k] / 4, r = e[k] % 4;
                // the lower corner of edge e[k]: r with a zero bit inserted at a
                const int lo = ((r >> a) << (a + 1)) | (r & ((1 << a) - 1));
                all = all && a != b && ((lo >> b) & 1) == side;
            }
            if (all) return true;
        }
    return false;
}

CubeCases build_cube_cases() {
    CubeCases cc;
    std::memset(&cc, 0, sizeof cc);
    for (int mask = 0; mask < 256; ++mask) {
        int succ[12];
        std::fill(succ, succ + 12, -1);
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 2; ++s) {
                int ring[4];
                face_ring(a, s, ring);
                auto in = [&](int i) { return (mask >> ring[(i + 4) % 4]) & 1; };
                for (int i = 0; i < 4; ++i) {
                    if (!in(i) || in(i - 1)) continue;  // not the first corner of an inside run
                    int j = i;
                    while (in(j + 1)) ++j;
                    succ[cube_edge(ring[(i + 3) % 4], ring[i])] = cube_edge(ring[j % 4], ring[(j + 1) % 4]);
                }
            }
        int n = 0;
        bool used[12] = {false};
        for (int first = 0; first < 12; ++first) {
            if (succ[first] < 0 || used[first]) continue;
            std::vector<int> loop;
            for (int e = first; !used[e]; e = succ[e]) {
                used[e] = true;
                loop.push_back(e);
            }
            const int m = (int)loop.size();
            int start = 0;
            for (int st = 0; st < m; ++st) {
                bool flat = false;
                for (int i = 1; i + 1 < m && !flat; ++i) {
                    const int tri[3] = {loop[st], loop[(st + i) % m], loop[(st + i + 1) % m]};
                    flat = edges_share_a_face(tri);
                }
                if (!flat) {
                    start = st;
                    break;
                }
            }
            for (int i = 1; i + 1 < m; ++i, ++n) {
                cc.t[mask][1 + 3 * n] = (uint8_t)loop[start];
                cc.t[mask][2 + 3 * n] = (uint8_t)loop[(start + i) % m];
                cc.t[mask][3 + 3 * n] = (uint8_t)loop[(start + i + 1) % m];
            }
        }
        cc.t[mask][0] = (uint8_t)n;
    }
    return cc;
}

const CubeCases& cube_cases() {
    static const CubeCases cc = build_cube_cases();
    return cc;
}

}  // namespace

extern "C" tsdf_status tsdf_mesh(tsdf_volume* v, float* triangles, int64_t capacity, int64_t* n_triangles) {
    return tsdf_mesh_ex(v, TSDF_MESH_CUBES, triangles, capacity, n_triangles);
}

extern "C" tsdf_status tsdf_mesh_ex(tsdf_volume* v, int32_t method, float* triangles, int64_t capacity,
                                    int64_t* n_triangles) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (method != TSDF_MESH_CUBES && method != TSDF_MESH_TETRAHEDRA)
        return fail(v, TSDF_ERR_INVALID_ARG, "mesh: unknown method");
    if (v->zoff_g != 0 || v->ng[2] != v->ngz_all) return fail(v, TSDF_ERR_INVALID_ARG, "mesh: needs a whole volume");
    if (!n_triangles || capacity < 0 || (capacity > 0 && !triangles))
        return fail(v, TSDF_ERR_INVALID_ARG, "mesh: need n_triangles, capacity >= 0 and a buffer for it");
    Temps t(v);
    const size_t nbt = (size_t)v->nb[0] * v->nb[1] * v->nb[2];
    uint32_t* list = (uint32_t*)t.get(nbt * sizeof(uint32_t));
    uint32_t* n_list = (uint32_t*)t.get(sizeof(uint32_t) + sizeof(unsigned long long) * 2);
    const size_t out_bytes = (size_t)capacity * 9 * sizeof(float);
    float* out = (float*)output(t, triangles, out_bytes);
    if (!list || !n_list || (capacity > 0 && !out)) return fail(v, TSDF_ERR_OOM, "mesh: scratch buffers");
    unsigned long long* count = reinterpret_cast<unsigned long long*>(n_list + 2);
    cudaError_t e = cudaMemsetAsync(n_list, 0, sizeof(uint32_t) + sizeof(unsigned long long) * 2, v->stream);
    if (e == cudaSuccess && method == TSDF_MESH_CUBES) e = tsdf::upload_cube_cases(cube_cases().t, v->stream);
    if (e == cudaSuccess)
        e = tsdf::launch_mesh(mesh_const(v), v->vol.F, v->vol.W, v->vol.summ, list, n_list, out,
                              (uint64_t)capacity, count, method == TSDF_MESH_CUBES, v->stream);
    unsigned long long total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, count, sizeof total, cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    if (e == cudaSuccess)
        e = finish(v, triangles, out, (size_t)std::min<int64_t>(capacity, (int64_t)total) * 9 * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    if (e != cudaSuccess) return cuda_fail(v, e, "mesh");
    *n_triangles = (int64_t)total;
    return TSDF_OK;
}

extern "C" tsdf_status tsdf_texture_layout(tsdf_volume* v, const float* triangles, int64_t n, float size_pixel,
                                           int32_t max_side, int32_t* wh, int64_t* offsets) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (n < 0 || n > (int64_t(1) << 31) || (n > 0 && (!triangles || !wh)) || !offsets ||
        !(size_pixel > 0.0f) || !std::isfinite(size_pixel) || max_side < 2 || max_side > 65536)
        return fail(v, TSDF_ERR_INVALID_ARG,
                    "texture layout: need 0 <= n <= 2^31, triangles, wh, offsets, size_pixel > 0, 2 <= max_side "
                    "<= 65536");
    Temps t(v);
    cudaError_t e = cudaSuccess;
    const float* d_tris = (const float*)input(v, t, triangles, (size_t)n * 9 * sizeof(float), e);
    int32_t* d_wh = (int32_t*)output(t, wh, (size_t)n * 2 * sizeof(int32_t));
    int64_t* d_off = (int64_t*)output(t, offsets, (size_t)(n + 1) * sizeof(int64_t));
    const int64_t nb = (n + 1023) / 1024;
    int64_t* scratch = (int64_t*)t.get((size_t)(nb + 1) * sizeof(int64_t));
    if ((n > 0 && (!d_tris || !d_wh)) || !d_off || !scratch) return fail(v, TSDF_ERR_OOM, "texture layout buffers");
    if (e == cudaSuccess) e = tsdf::launch_texture_layout(d_tris, n, size_pixel, max_side, d_wh, d_off, scratch, v->stream);
    if (e == cudaSuccess) e = finish(v, wh, d_wh, (size_t)n * 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = finish(v, offsets, d_off, (size_t)(n + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "texture layout");
}

extern "C" tsdf_status tsdf_texture_fill(tsdf_volume* v, const float* triangles, int64_t n, const int32_t* wh,
                                         const int64_t* offsets, uint32_t* texels) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (v->zoff_c != 0 || v->nc[2] != v->ncz_all)
        return fail(v, TSDF_ERR_INVALID_ARG, "texture fill: needs a whole volume");
    if (n < 0 || n > (int64_t(1) << 31) || (n > 0 && (!triangles || !wh || !offsets || !texels)))
        return fail(v, TSDF_ERR_INVALID_ARG, "texture fill: need triangles, wh, offsets and texels");
    if (n == 0) return TSDF_OK;
    int64_t total = 0;
    cudaError_t e = cudaSuccess;
    if (is_device_ptr(offsets)) {
        e = cudaMemcpyAsync(&total, offsets + n, sizeof total, cudaMemcpyDeviceToHost, v->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
        if (e != cudaSuccess) return cuda_fail(v, e, "texture fill");
    } else {
        total = offsets[n];
    }
    if (total < 0) return fail(v, TSDF_ERR_INVALID_ARG, "texture fill: negative texel total");
    Temps t(v);
    const float* d_tris = (const float*)input(v, t, triangles, (size_t)n * 9 * sizeof(float), e);
    const int32_t* d_wh = (const int32_t*)input(v, t, wh, (size_t)n * 2 * sizeof(int32_t), e);
    const int64_t* d_off = (const int64_t*)input(v, t, offsets, (size_t)(n + 1) * sizeof(int64_t), e);
    uint32_t* d_tex = (uint32_t*)output(t, texels, (size_t)total * sizeof(uint32_t));
    if (!d_tris || !d_wh || !d_off || (total > 0 && !d_tex)) return fail(v, TSDF_ERR_OOM, "texture fill buffers");
    tsdf::ColourConst c;
    std::memset(&c, 0, sizeof c);
    for (int a = 0; a < 3; ++a) {
        c.nc[a] = v->nc[a];
        c.ncb[a] = v->ncb[a];
        c.origin[a] = v->origin[a];
    }
    c.s_c = v->s_c;
    c.inv_sc = (float)(1.0 / (double)v->s_c);
    if (e == cudaSuccess) e = tsdf::launch_texture_fill(c, v->vol.C, d_tris, n, d_wh, d_off, total, d_tex, v->stream);
    if (e == cudaSuccess) e = finish(v, texels, d_tex, (size_t)total * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    return e == cudaSuccess ? TSDF_OK : cuda_fail(v, e, "texture fill");
}
