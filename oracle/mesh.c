/*
 * CPU ORACLE of mesh extraction from the geometry volume and of the
 * per-polygon 2D texture maps sampled from the colour volume (Section IV.C
 * "Mesh Extraction and Simplification" and Section IV.D "Texture
 * Generation", Eq. 11-14).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests may load this file's library.
 * The CUDA path shares no code with it.
 *
 * Binary32 with the operation order written here (-ffp-contract=off; fmaf is
 * the correctly rounded fused multiply-add).
 *
 * Mesh: the zero level set of the TSDF by marching cubes (orc_mesh_cubes,
 * described at its definition below) or, as an option, by marching
 * tetrahedra (orc_mesh).  Marching tetrahedra:  a cell is the
 * cube of eight neighbouring geometry voxels (x..x+1, y..y+1, z..z+1), corner
 * k = (k & 1, (k >> 1) & 1, k >> 2); it is meshed only when all eight corners
 * are observed (w > 0).  The cell is split into six tetrahedra along its main
 * diagonal (corner 0 to corner 7): for each ordering (a0, a1, a2) of the axes,
 * in the order (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x), the
 * tetrahedron 0, 0 + a0, 0 + a0 + a1, 7.  This split is the same on the shared
 * face of two neighbouring cells, so the surface has no cracks.  A corner is
 * inside when F < 0.  A tetrahedron with one corner on its own side gives the
 * triangle on the three edges from that corner (the other corners in
 * tetrahedron order); one with two inside corners i1, i2 and two outside
 * corners o1, o2 (tetrahedron order) gives the quad on edges (i1,o1),
 * (i1,o2), (i2,o2), (i2,o1), split into the triangles ((i1,o1), (i1,o2),
 * (i2,o2)) and ((i1,o1), (i2,o2), (i2,o1)).  The vertex on edge (p, q), with p
 * the corner of lower linear voxel index: t = F_p / (F_p - F_q), v = fmaf(t,
 * P_q - P_p, P_p) per axis, P the voxel centre fmaf(i + 1/2, s_g, origin).
 * Orientation: with n = (v1 - v0) x (v2 - v0) (each component a product minus
 * a product) and d = P_out - P_in (the first outside and first inside corner
 * of the tetrahedron), a triangle with fmaf(n_x, d_x, fmaf(n_y, d_y, n_z d_z))
 * < 0 has v1 and v2 swapped, so normals point to free space.  Triangles come
 * in cell order (linear index, x fastest), tetrahedron order, triangle order.
 *
 * Texture maps (Eq. 11-14): for a triangle (V_a, V_b, V_c) and pixel size s,
 * w = max(2, floor(|V_a V_b| / s + 1/2)) and h = max(2, floor(|V_a V_c| / s + 1/2))
 * (Eq. 11-12 rounded to the nearest texel count), capped at max_side
 * (|.| = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz dz)))); green = (V_b -
 * V_a) / (w - 1), blue = (V_c - V_a) / (h - 1) per axis; texel (i, j), i the
 * column along green and j the row along blue, lies at p = fmaf(j, blue,
 * fmaf(i, green, V_a)) (the worked example: the pixel two columns and three
 * rows from V_a is V_a + 2 green + 3 blue).  Its colour is the trilinear
 * interpolation of the colour volume at p over the observed colour voxels
 * only (g = fmaf(p - origin, 1/s_c, -1/2), i0 = floor(g), f = g - i0, corner
 * weight ((x ? f_x : 1 - f_x) (y ? f_y : 1 - f_y)) (z ? f_z : 1 - f_z), corners
 * in order k = 0..7 accumulated with fmaf into per-channel sums and a weight
 * sum; corners outside the volume or with colour weight 0 are left out),
 * each channel floor(sum / wsum + 1/2) as 8 bits and alpha 255; a texel
 * with no observed corner (or wsum = 0) is 0.  Maps are row-major, h rows of
 * w texels, packed R | G << 8 | B << 16 | A << 24, one after another in
 * triangle order.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int32_t ng[3];
    float s_g;
    float origin[3];
    const float* F;
    const uint8_t* W;
} orc_mesh_volume;

static const int TET_AXES[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static float centre_of(const orc_mesh_volume* v, int a, int i) { return fmaf((float)i + 0.5f, v->s_g, v->origin[a]); }

/* Vertex on the edge between cell corners a and b. */
static void edge_vertex(const orc_mesh_volume* v, const int base[3], const float Fc[8], int a, int b, float out[3]) {
    /* corner index order equals linear voxel index order within a cell */
    int p = a < b ? a : b, q = a < b ? b : a;
    float t = Fc[p] / (Fc[p] - Fc[q]);
    for (int ax = 0; ax < 3; ++ax) {
        float Pp = centre_of(v, ax, base[ax] + ((p >> ax) & 1));
        float Pq = centre_of(v, ax, base[ax] + ((q >> ax) & 1));
        out[ax] = fmaf(t, Pq - Pp, Pp);
    }
}

static void emit(const orc_mesh_volume* v, const int base[3], const float tri[9], int cin, int cout, float* out) {
    float e1[3], e2[3], n[3], d[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = tri[3 + a] - tri[a];
        e2[a] = tri[6 + a] - tri[a];
        d[a] = centre_of(v, a, base[a] + ((cout >> a) & 1)) - centre_of(v, a, base[a] + ((cin >> a) & 1));
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    float dot = fmaf(n[0], d[0], fmaf(n[1], d[1], n[2] * d[2]));
    memcpy(out, tri, 9 * sizeof(float));
    if (dot < 0.0f) {
        memcpy(out + 3, tri + 6, 3 * sizeof(float));
        memcpy(out + 6, tri + 3, 3 * sizeof(float));
    }
}

/* Triangles of one cell into out (up to 12 x 9 floats); returns the count. */
static int cell_triangles(const orc_mesh_volume* v, int x, int y, int z, float* out) {
    const int base[3] = {x, y, z};
    float Fc[8];
    for (int k = 0; k < 8; ++k) {
        size_t idx = ((size_t)(z + (k >> 2)) * v->ng[1] + (y + ((k >> 1) & 1))) * v->ng[0] + (x + (k & 1));
        if (v->W[idx] == 0) return 0;
        Fc[k] = v->F[idx];
    }
    int n = 0;
    for (int t = 0; t < 6; ++t) {
        int c[4];
        c[0] = 0;
        c[1] = 1 << TET_AXES[t][0];
        c[2] = c[1] | (1 << TET_AXES[t][1]);
        c[3] = 7;
        int ins[4], outs[4], ni = 0, no = 0;
        for (int k = 0; k < 4; ++k) {
            if (Fc[c[k]] < 0.0f) ins[ni++] = c[k];
            else outs[no++] = c[k];
        }
        if (ni == 0 || no == 0) continue;
        float tri[9];
        if (ni == 1 || no == 1) {
            int lone = ni == 1 ? ins[0] : outs[0];
            const int* others = ni == 1 ? outs : ins;
            for (int e = 0; e < 3; ++e) edge_vertex(v, base, Fc, lone, others[e], tri + 3 * e);
            emit(v, base, tri, ins[0], outs[0], out + 9 * n++);
        } else {
            float q[4][3];
            edge_vertex(v, base, Fc, ins[0], outs[0], q[0]);
            edge_vertex(v, base, Fc, ins[0], outs[1], q[1]);
            edge_vertex(v, base, Fc, ins[1], outs[1], q[2]);
            edge_vertex(v, base, Fc, ins[1], outs[0], q[3]);
            memcpy(tri, q[0], 12); memcpy(tri + 3, q[1], 12); memcpy(tri + 6, q[2], 12);
            emit(v, base, tri, ins[0], outs[0], out + 9 * n++);
            memcpy(tri, q[0], 12); memcpy(tri + 3, q[2], 12); memcpy(tri + 6, q[3], 12);
            emit(v, base, tri, ins[0], outs[0], out + 9 * n++);
        }
    }
    return n;
}

/* ---------------------------------------------------- marching cubes ---- */
/* Marching cubes (Section IV.C), written as its definition, cell by cell,
 * without a case table.  Cells, corners, "inside" (F < 0), observed cells and
 * the vertex on an edge are as above.  The twelve edges of a cell are
 * numbered 4 a + r: a the axis along which the edge runs, r the rank of its
 * lower corner among the four corners whose bit a is 0.
 *
 * The surface's boundary on each face of the cell: with the face's corners
 * c0..c3 taken counter-clockwise about the face's outward normal and e_i the
 * edge from c_i to c_(i+1), every maximal run c_i..c_j of consecutive inside
 * corners is cut off by one segment from edge e_(i-1) to edge e_j.  A face
 * with two diagonal inside corners therefore separates them (the reading of
 * the face ambiguity taken here; neighbouring cells see the same face alike,
 * so the surface has no cracks).  Every crossing edge then starts one segment
 * and ends one, and the segments form closed loops; the loops are taken in
 * the order of their lowest edge and each is triangulated as a fan from that
 * edge's vertex, along the segments' direction: (v0, v1, v2), (v0, v2, v3),
 * ...  With this direction the triangles' normals (v1 - v0) x (v2 - v0) point
 * to the outside (F >= 0).  A loop that crosses one face twice would give,
 * fanned from some vertices, a triangle lying flat in that face (and the
 * neighbouring cell the same triangle reversed); the fan therefore starts at
 * the first vertex, in loop order from the lowest edge, whose fan has no
 * triangle with all three vertices on edges of one face (the lowest edge's
 * vertex when none qualifies).  Triangles come in cell order (linear index,
 * x fastest), loop order, fan order. */
static const int FACE_CCW[6][4] = {
    {0, 4, 6, 2},  /* x = 0, normal -x */
    {1, 3, 7, 5},  /* x = 1, normal +x */
    {0, 1, 5, 4},  /* y = 0, normal -y */
    {2, 6, 7, 3},  /* y = 1, normal +y */
    {0, 2, 3, 1},  /* z = 0, normal -z */
    {4, 5, 7, 6},  /* z = 1, normal +z */
};

/* Edge number of the cell edge between corners p and q (one bit apart). */
static int edge_of(int p, int q) {
    int lo = p < q ? p : q, d = p ^ q, a = d == 1 ? 0 : (d == 2 ? 1 : 2), r = 0;
    for (int c = 0; c < lo; ++c)
        if (!((c >> a) & 1)) ++r;
    return 4 * a + r;
}

/* The two corners (lower first) of edge e. */
static void edge_corners(int e, int* p, int* q) {
    int a = e / 4, r = e % 4;
    for (int c = 0; c < 8; ++c)
        if (!((c >> a) & 1) && r-- == 0) {
            *p = c;
            *q = c | (1 << a);
            return;
        }
}

/* Whether edges e0, e1, e2 all lie in one face of the cell.  The edge with
 * lower corner p along axis a lies in the faces (b, bit b of p), b != a. */
static int on_one_face(int e0, int e1, int e2) {
    const int es[3] = {e0, e1, e2};
    for (int b = 0; b < 3; ++b)
        for (int side = 0; side < 2; ++side) {
            int all = 1;
            for (int k = 0; k < 3 && all; ++k) {
                int p, q;
                edge_corners(es[k], &p, &q);
                all = (es[k] / 4 != b) && (((p >> b) & 1) == side);
            }
            if (all) return 1;
        }
    return 0;
}

static int cell_cubes(const orc_mesh_volume* v, int x, int y, int z, float* out) {
    const int base[3] = {x, y, z};
    float Fc[8];
    int inside = 0;
    for (int k = 0; k < 8; ++k) {
        size_t idx = ((size_t)(z + (k >> 2)) * v->ng[1] + (y + ((k >> 1) & 1))) * v->ng[0] + (x + (k & 1));
        if (v->W[idx] == 0) return 0;
        Fc[k] = v->F[idx];
        if (Fc[k] < 0.0f) inside |= 1 << k;
    }
    if (inside == 0 || inside == 255) return 0;
    int next[12];
    for (int e = 0; e < 12; ++e) next[e] = -1;
    for (int f = 0; f < 6; ++f) {
        const int* c = FACE_CCW[f];
        for (int i = 0; i < 4; ++i) {
            int in_i = (inside >> c[i]) & 1, in_prev = (inside >> c[(i + 3) % 4]) & 1;
            if (!in_i || in_prev) continue;  /* i starts a run of inside corners */
            int j = i;
            while ((inside >> c[(j + 1) % 4]) & 1) j = (j + 1) % 4;
            next[edge_of(c[(i + 3) % 4], c[i])] = edge_of(c[j], c[(j + 1) % 4]);
        }
    }
    int n = 0, seen[12] = {0};
    for (int e0 = 0; e0 < 12; ++e0) {
        if (next[e0] < 0 || seen[e0]) continue;
        int loop[12], m = 0;
        for (int e = e0; !seen[e]; e = next[e]) {
            seen[e] = 1;
            loop[m++] = e;
        }
        float vert[12][3];
        for (int i = 0; i < m; ++i) {
            int p, q;
            edge_corners(loop[i], &p, &q);
            edge_vertex(v, base, Fc, p, q, vert[i]);
        }
        int s0 = 0;
        for (int s = 0; s < m; ++s) {
            int flat = 0;
            for (int i = 1; i + 1 < m && !flat; ++i)
                flat = on_one_face(loop[s], loop[(s + i) % m], loop[(s + i + 1) % m]);
            if (!flat) {
                s0 = s;
                break;
            }
        }
        for (int i = 1; i + 1 < m; ++i, ++n) {
            memcpy(out + 9 * n, vert[s0], 12);
            memcpy(out + 9 * n + 3, vert[(s0 + i) % m], 12);
            memcpy(out + 9 * n + 6, vert[(s0 + i + 1) % m], 12);
        }
    }
    return n;
}

/* Marching-cubes mesh: writes up to cap triangles (9 floats each) to tris
 * (may be NULL) and returns the total number of triangles. */
long long orc_mesh_cubes(const orc_mesh_volume* v, float* tris, long long cap) {
    long long n = 0;
    float buf[12 * 9];
    for (int z = 0; z + 1 < v->ng[2]; ++z)
        for (int y = 0; y + 1 < v->ng[1]; ++y)
            for (int x = 0; x + 1 < v->ng[0]; ++x) {
                int m = cell_cubes(v, x, y, z, buf);
                for (int i = 0; i < m; ++i, ++n)
                    if (tris && n < cap) memcpy(tris + 9 * n, buf + 9 * i, 9 * sizeof(float));
            }
    return n;
}

/* Extract the mesh: writes up to cap triangles (9 floats each) to tris (may
 * be NULL) and returns the total number of triangles. */
long long orc_mesh(const orc_mesh_volume* v, float* tris, long long cap) {
    long long n = 0;
    float buf[12 * 9];
    for (int z = 0; z + 1 < v->ng[2]; ++z)
        for (int y = 0; y + 1 < v->ng[1]; ++y)
            for (int x = 0; x + 1 < v->ng[0]; ++x) {
                int m = cell_triangles(v, x, y, z, buf);
                for (int i = 0; i < m; ++i, ++n)
                    if (tris && n < cap) memcpy(tris + 9 * n, buf + 9 * i, 9 * sizeof(float));
            }
    return n;
}

/* ----------------------------------------------------------- texture ---- */
typedef struct {
    int32_t nc[3];
    float s_c;
    float origin[3];
    const uint32_t* C;
} orc_colour_volume;

static int side(float dist, float size_pixel, int max_side) {
    float q = floorf(dist / size_pixel + 0.5f);
    if (!(q >= 2.0f)) return 2;  /* also NaN */
    if (q > (float)max_side) return max_side;
    return (int)q;
}

static float length3(const float d[3]) { return sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]))); }

/* Eq. 11-12: texture map sizes (w, h) of n triangles; returns the texel total. */
long long orc_texture_sizes(const float* tris, long long n, float size_pixel, int max_side, int32_t* wh) {
    long long total = 0;
    for (long long i = 0; i < n; ++i) {
        const float* T = tris + 9 * i;
        float ab[3], ac[3];
        for (int a = 0; a < 3; ++a) {
            ab[a] = T[3 + a] - T[a];
            ac[a] = T[6 + a] - T[a];
        }
        wh[2 * i] = side(length3(ab), size_pixel, max_side);
        wh[2 * i + 1] = side(length3(ac), size_pixel, max_side);
        total += (long long)wh[2 * i] * wh[2 * i + 1];
    }
    return total;
}

static uint32_t texel(const orc_colour_volume* cv, float inv_sc, const float p[3]) {
    float g[3], f[3];
    int i0[3];
    for (int a = 0; a < 3; ++a) {
        g[a] = fmaf(p[a] - cv->origin[a], inv_sc, -0.5f);
        float fl = floorf(g[a]);
        if (!(fl >= -1.0f) || !(fl <= (float)cv->nc[a])) return 0u;  /* no corner can be inside */
        i0[a] = (int)fl;
        f[a] = g[a] - fl;
    }
    float acc[3] = {0.0f, 0.0f, 0.0f}, wsum = 0.0f;
    for (int k = 0; k < 8; ++k) {
        int x = i0[0] + (k & 1), y = i0[1] + ((k >> 1) & 1), z = i0[2] + (k >> 2);
        if (x < 0 || y < 0 || z < 0 || x >= cv->nc[0] || y >= cv->nc[1] || z >= cv->nc[2]) continue;
        uint32_t c = cv->C[((size_t)z * cv->nc[1] + y) * cv->nc[0] + x];
        if ((c >> 24) == 0u) continue;
        float wgt = ((k & 1) ? f[0] : 1.0f - f[0]) * (((k >> 1) & 1) ? f[1] : 1.0f - f[1]);
        wgt = wgt * ((k >> 2) ? f[2] : 1.0f - f[2]);
        for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(wgt, (float)((c >> (8 * ch)) & 0xFFu), acc[ch]);
        wsum = wsum + wgt;
    }
    if (!(wsum > 0.0f)) return 0u;
    uint32_t out = 255u << 24;
    for (int ch = 0; ch < 3; ++ch) {
        float val = floorf(acc[ch] / wsum + 0.5f);
        uint32_t u = val <= 0.0f ? 0u : (val >= 255.0f ? 255u : (uint32_t)val);
        out |= u << (8 * ch);
    }
    return out;
}

/* Eq. 13-14 and the texel lookup: fill the maps of n triangles (sizes wh,
 * texel offsets off[n]) into texels. */
void orc_texture_fill(const orc_colour_volume* cv, const float* tris, long long n, const int32_t* wh,
                      const int64_t* off, uint32_t* texels) {
    const float inv_sc = (float)(1.0 / (double)cv->s_c);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < n; ++t) {
        const float* T = tris + 9 * t;
        const int w = wh[2 * t], h = wh[2 * t + 1];
        float green[3], blue[3];
        for (int a = 0; a < 3; ++a) {
            green[a] = (T[3 + a] - T[a]) / (float)(w - 1);
            blue[a] = (T[6 + a] - T[a]) / (float)(h - 1);
        }
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                float p[3];
                for (int a = 0; a < 3; ++a) p[a] = fmaf((float)j, blue[a], fmaf((float)i, green[a], T[a]));
                texels[off[t] + (int64_t)j * w + i] = texel(cv, inv_sc, p);
            }
    }
}

int orc_mesh_sizes(int which) { return which == 0 ? (int)sizeof(orc_mesh_volume) : (int)sizeof(orc_colour_volume); }
