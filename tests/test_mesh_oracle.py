"""Pins of the mesh and texture-map oracle (oracle/mesh.c).

Mesh (the TSDF zero level set by marching cubes, Section IV.C, and by
marching tetrahedra as an option): volumes written from analytic signed
distances; a plane's vertices lie on the plane and tile its cross-section
exactly, a sphere gives a closed, consistently oriented surface of Euler
characteristic 2 on the sphere, unobserved cells give nothing.  Marching
cubes alone: single cells whose surface is worked out by hand (the corner cut
off by one triangle, a quad, the separated corners of an ambiguous face, the
hexagon of its complement), and random fields full of ambiguous faces that
must still give a closed, consistently oriented surface.

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


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
def test_plane_vertices_on_the_plane_and_area_exact(oracle_lib, method):
    z0 = -0.0731
    _, _, z = centres(N, S_G)
    F, W = field(z - z0)
    T = oracle.mesh(F, W, S_G, ORIGIN, method)
    assert len(T) > 0
    np.testing.assert_allclose(T[..., 2], z0, atol=1e-6)
    n = tri_normals(T)
    area = 0.5 * np.linalg.norm(n, axis=1)
    # free space is above (F > 0): normals point up
    assert np.all(n[area > 1e-12, 2] > 0)
    np.testing.assert_allclose(area.sum(), ((N - 1) * S_G) ** 2, rtol=1e-5)


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
def test_tilted_plane(oracle_lib, method):
    nrm = np.array([0.3, -0.5, 0.81])
    nrm /= np.linalg.norm(nrm)
    x, y, z = centres(N, S_G)
    F, W = field(nrm[0] * x + nrm[1] * y + nrm[2] * z - 0.013)
    T = oracle.mesh(F, W, S_G, ORIGIN, method).astype(np.float64)
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


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
def test_sphere_is_closed_oriented_and_on_the_sphere(oracle_lib, method):
    c, r = np.array([0.031, -0.022, 0.017]), 0.29
    x, y, z = centres(N, S_G)
    F, W = field(np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r)
    T = oracle.mesh(F, W, S_G, ORIGIN, method)
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


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
def test_unobserved_cells_give_no_triangles(oracle_lib, method):
    _, _, z = centres(N, S_G)
    F, W = field(z - 0.0123)
    W[:, :, : N // 2] = 0
    T = oracle.mesh(F, W, S_G, ORIGIN, method)
    assert len(T) > 0 and T[..., 0].max() >= -0.5 and T[..., 0].min() >= ORIGIN[0] + (N // 2 + 0.5) * S_G - 1e-6
    assert len(oracle.mesh(F, np.zeros_like(W), S_G, ORIGIN, method)) == 0


# ------------------------------------------------------ marching cubes only --
def one_cell(inside):
    """A single observed cell (2 x 2 x 2 voxels of edge 1, origin 0) whose
    corners k = x + 2 y + 4 z in `inside` hold F = -0.5, the others +0.5, so
    every crossing sits at the middle of its edge."""
    F = np.full((2, 2, 2), 0.5, np.float32)
    for k in inside:
        F[k >> 2, (k >> 1) & 1, k & 1] = -0.5
    return oracle.mesh(F, np.ones((2, 2, 2), np.uint8), 1.0, (-0.5, -0.5, -0.5), "cubes")


def corner(k):
    return np.array([k & 1, (k >> 1) & 1, k >> 2], np.float64)


def midpoints(k):
    """Midpoints of the three edges at corner k."""
    c = corner(k)
    return {tuple(c + 0.5 * (1 - 2 * c[a]) * np.eye(3)[a]) for a in range(3)}


def test_cube_single_corner_and_edge(oracle_lib):
    T = one_cell([0])
    assert len(T) == 1
    assert {tuple(v) for v in T[0].astype(np.float64)} == midpoints(0)
    assert np.all(tri_normals(T)[0] > 0)  # away from the inside corner 0, toward (1, 1, 1)
    T = one_cell([0, 1])  # the quad on the four edges leaving the x edge (0, 1)
    assert len(T) == 2
    verts = {tuple(v) for v in T.reshape(-1, 3).astype(np.float64)}
    assert verts == {(0, 0.5, 0), (0, 0, 0.5), (1, 0.5, 0), (1, 0, 0.5)}
    n = tri_normals(T)
    assert np.all(n[:, 0] == 0) and np.all(n[:, 1] > 0) and np.all(n[:, 2] > 0)


@pytest.mark.parametrize("inside,groups", [
    ([0, 3], [[0], [3]]),              # diagonal of the face z = 0: the corners stay apart
    ([0, 7], [[0], [7]]),              # body diagonal
    ([0, 3, 5, 6], [[0], [3], [5], [6]]),  # every face ambiguous
])
def test_cube_ambiguous_faces_separate_the_inside_corners(oracle_lib, inside, groups):
    T = one_cell(inside)
    assert len(T) == len(groups)
    for tri in T:
        vs = {tuple(v) for v in tri.astype(np.float64)}
        k = [g[0] for g in groups if vs == midpoints(g[0])]
        assert len(k) == 1  # each triangle cuts off exactly one inside corner
        assert np.dot(tri_normals(tri[None])[0], tri.astype(np.float64).mean(0) - corner(k[0])) > 0


def test_cube_complement_of_a_face_diagonal_is_a_hexagon(oracle_lib):
    """Outside corners 0 and 3 (a diagonal of face z = 0), the rest inside:
    that face separates its inside corners 1 and 2, so the outside corners stay
    connected and the surface is one hexagon on the edges (0,1), (1,3), (3,2),
    (2,0), (0,4), (3,7): four triangles, normals toward the outside corners."""
    T = one_cell([1, 2, 4, 5, 6, 7])
    assert len(T) == 4
    verts = {tuple(v) for v in T.reshape(-1, 3).astype(np.float64)}
    assert verts == {(0.5, 0, 0), (1, 0.5, 0), (0.5, 1, 0), (0, 0.5, 0), (0, 0, 0.5), (1, 1, 0.5)}
    for tri in T.astype(np.float64):
        n = tri_normals(tri[None])[0]
        m = tri.mean(0)
        toward = corner(0) if np.linalg.norm(m - corner(0)) < np.linalg.norm(m - corner(3)) else corner(3)
        assert np.dot(n, toward - m) >= 0


@pytest.mark.parametrize("seed", range(4))
def test_cube_random_fields_give_closed_oriented_surfaces(oracle_lib, seed):
    """Random corner values (many ambiguous faces) inside a positive shell:
    every surface edge is shared by exactly two triangles, once in each
    direction, so neighbouring cells resolve their shared faces alike."""
    rng = np.random.default_rng(seed)
    n = 12
    F = rng.uniform(-1, 1, size=(n, n, n)).astype(np.float32)
    F[0], F[-1], F[:, 0], F[:, -1], F[:, :, 0], F[:, :, -1] = 1, 1, 1, 1, 1, 1
    T = oracle.mesh(F, np.ones_like(F, np.uint8), 0.1, (0.0, 0.0, 0.0), "cubes")
    assert len(T) > 200
    _, und, directed = edge_counts(T)
    assert all(v == 2 for v in und.values())
    assert all(v == 1 for v in directed.values())


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
