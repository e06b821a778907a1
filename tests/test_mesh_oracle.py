"""Pins of the mesh and texture-map oracle (oracle/mesh.c).

Mesh (marching tetrahedra of the TSDF zero level set): volumes written from
analytic signed distances; a plane's vertices lie on the plane and tile its
cross-section exactly, a sphere gives a closed, consistently oriented surface
of Euler characteristic 2 on the sphere, unobserved cells give nothing.

Texture maps (Section IV.D, Eq. 11-14): map sizes in closed form, the worked
example of the paper (tests/golden/texture_worked_example.json) through a
colour volume that encodes position, constant colour, and unobserved colour
voxels left out of the interpolation.
"""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
N = 40
S_G = 1.0 / N
MU = 3 * S_G
ORIGIN = (-0.5, -0.5, -0.5)


def centres(n, s):
    c = ORIGIN[0] + (np.arange(n, dtype=np.float64) + 0.5) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


def field(sd):
    F = np.clip(sd / MU, -1.0, 1.0).astype(np.float32)
    return F, np.ones_like(F, np.uint8)


def tri_normals(T):
    T = T.astype(np.float64)
    return np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])


def test_plane_vertices_on_the_plane_and_area_exact(oracle_lib):
    z0 = -0.0731
    _, _, z = centres(N, S_G)
    F, W = field(z - z0)
    T = oracle.mesh(F, W, S_G, ORIGIN)
    assert len(T) > 0
    np.testing.assert_allclose(T[..., 2], z0, atol=1e-6)
    n = tri_normals(T)
    area = 0.5 * np.linalg.norm(n, axis=1)
    # free space is above (F > 0): normals point up
    assert np.all(n[area > 1e-12, 2] > 0)
    np.testing.assert_allclose(area.sum(), ((N - 1) * S_G) ** 2, rtol=1e-5)


def test_tilted_plane(oracle_lib):
    nrm = np.array([0.3, -0.5, 0.81])
    nrm /= np.linalg.norm(nrm)
    x, y, z = centres(N, S_G)
    F, W = field(nrm[0] * x + nrm[1] * y + nrm[2] * z - 0.013)
    T = oracle.mesh(F, W, S_G, ORIGIN).astype(np.float64)
    np.testing.assert_allclose(T @ nrm, 0.013, atol=2e-6)
    n = tri_normals(T)
    big = np.linalg.norm(n, axis=1) > 1e-10
    assert np.all(n[big] @ nrm > 0)


def edge_counts(T):
    key = {}
    vid = np.unique(T.reshape(-1, 3).view(np.dtype((np.void, 12))), return_inverse=True)[1].reshape(-1, 3)
    directed = {}
    for a, b, c in vid:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(u, v)] = directed.get((u, v), 0) + 1
            e = (min(u, v), max(u, v))
            key[e] = key.get(e, 0) + 1
    return vid, key, directed


def test_sphere_is_closed_oriented_and_on_the_sphere(oracle_lib):
    c, r = np.array([0.031, -0.022, 0.017]), 0.29
    x, y, z = centres(N, S_G)
    F, W = field(np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r)
    T = oracle.mesh(F, W, S_G, ORIGIN)
    V = T.reshape(-1, 3).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(V - c, axis=1), r, atol=0.05 * S_G)
    vid, und, directed = edge_counts(T)
    assert all(v == 2 for v in und.values())              # closed 2-manifold
    assert all(v == 1 for v in directed.values())         # consistent orientation
    nverts = len(np.unique(vid))
    assert nverts - len(und) + len(T) == 2                # Euler characteristic of a sphere
    n = tri_normals(T)
    big = np.linalg.norm(n, axis=1) > 1e-12
    out = ((T.astype(np.float64).mean(axis=1) - c) * n).sum(axis=1)
    assert np.all(out[big] > 0)                           # normals point to free space (outside)


def test_unobserved_cells_give_no_triangles(oracle_lib):
    _, _, z = centres(N, S_G)
    F, W = field(z - 0.0123)
    W[:, :, : N // 2] = 0
    T = oracle.mesh(F, W, S_G, ORIGIN)
    assert len(T) > 0 and T[..., 0].max() >= -0.5 and T[..., 0].min() >= ORIGIN[0] + (N // 2 + 0.5) * S_G - 1e-6
    assert len(oracle.mesh(F, np.zeros_like(W), S_G, ORIGIN)) == 0


# ---------------------------------------------------------------- texture --
NC = 64
S_C = 1.0 / NC


def ramp_colours():
    """Colour volume whose channels are affine in the voxel index: R = 10 + 3 kx,
    G = 20 + 2 ky, B = 5 + 3 kz (so trilinear interpolation is exact)."""
    k = np.arange(NC, dtype=np.uint32)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    return ((10 + 3 * kx) | ((20 + 2 * ky) << 8) | ((5 + 3 * kz) << 16) | (1 << 24)).astype(np.uint32)


def ramp_at(p):
    g = (np.asarray(p, np.float64) - np.asarray(ORIGIN)) / S_C - 0.5
    return np.array([10 + 3 * g[..., 0], 20 + 2 * g[..., 1], 5 + 3 * g[..., 2]])


def unpack(t):
    return np.stack([(t >> (8 * c)) & 0xFF for c in range(4)], -1).astype(np.int64)


def test_worked_example_of_the_paper(oracle_lib):
    g = json.load(open(os.path.join(HERE, "golden", "texture_worked_example.json")))
    tri = np.array([g["V_a"], g["V_b"], g["V_c"]], np.float32)[None]
    wh, off, tex = oracle.texture_maps(tri, ramp_colours(), S_C, ORIGIN, g["size_pixel"])
    assert tuple(wh[0]) == (g["w"], g["h"])
    i, j = g["texel"]
    texel = unpack(tex[off[0] + j * g["w"] + i])
    want = ramp_at(g["position"])
    assert texel[3] == 255
    np.testing.assert_array_equal(texel[:3], np.floor(want + 0.5).astype(np.int64))
    # every texel of the map follows V_a + i green + j blue
    ii, jj = np.meshgrid(np.arange(g["w"]), np.arange(g["h"]))
    Va, Vb, Vc = (np.array(g[k]) for k in ("V_a", "V_b", "V_c"))
    P = Va + ii[..., None] * (Vb - Va) / (g["w"] - 1) + jj[..., None] * (Vc - Va) / (g["h"] - 1)
    val = np.moveaxis(ramp_at(P), 0, -1) + 0.5
    all_want = np.floor(val).astype(np.int64)
    got = unpack(tex[off[0]:off[1]].reshape(g["h"], g["w"]))
    # a value within binary32 rounding of a rounding tie may round either way
    tie = np.abs(val - np.round(val)) < 1e-4
    assert tie.mean() < 0.5
    np.testing.assert_array_equal(got[..., :3][~tie], all_want[~tie])
    assert np.all(np.abs(got[..., :3] - all_want)[tie] <= 1)


def test_map_sizes_closed_form(oracle_lib):
    rng = np.random.default_rng(2)
    tris = rng.uniform(-0.3, 0.3, size=(200, 3, 3)).astype(np.float32)
    s = 0.013
    wh, off, _ = oracle.texture_maps(tris, ramp_colours(), S_C, ORIGIN, s)
    T = tris.astype(np.float64)
    w = np.maximum(2, np.floor(np.linalg.norm(T[:, 1] - T[:, 0], axis=1) / s + 0.5))
    h = np.maximum(2, np.floor(np.linalg.norm(T[:, 2] - T[:, 0], axis=1) / s + 0.5))
    np.testing.assert_array_equal(wh[:, 0], w)
    np.testing.assert_array_equal(wh[:, 1], h)
    assert off[-1] == int((w * h).sum())


def test_constant_colour_and_unobserved_voxels(oracle_lib):
    rng = np.random.default_rng(5)
    tris = rng.uniform(-0.25, 0.25, size=(50, 3, 3)).astype(np.float32)
    col = np.uint32(77 | (140 << 8) | (201 << 16) | (9 << 24))
    C = np.full((NC, NC, NC), col, np.uint32)
    # unobserved voxels carry a different colour and weight 0: they must not leak
    C[:, :, NC // 2:] = np.uint32(1 | (2 << 8) | (3 << 16))
    _, _, tex = oracle.texture_maps(tris, C, S_C, ORIGIN, 0.01)
    t = unpack(tex)
    seen = t[:, 3] == 255
    assert seen.sum() > 1000 and (~seen).sum() > 1000
    np.testing.assert_array_equal(t[seen, :3], np.broadcast_to([77, 140, 201], (seen.sum(), 3)))
    assert np.all(tex[~seen] == 0)
