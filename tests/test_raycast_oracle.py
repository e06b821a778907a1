"""Pins of the ray-casting oracle (oracle/raycast.c) against closed forms.

Volumes are written directly from analytic signed distances, so the expected
hits are known without the oracle: a plane seen from above (every ray hits
the plane; range, normal and colour voxel in closed form), a sphere (hits on
the sphere, radial normals), and the cases that must miss (unobserved
volume, camera looking away, camera inside the solid).
"""
import math

import numpy as np
import pytest

import oracle

N = 64            # geometry voxels per edge (1 m cube)
S_G = 1.0 / N
MU = 3 * S_G
ORIGIN = (-0.5, -0.5, -0.5)
K = np.array([[120.0, 0.0, 39.5], [0.0, 120.0, 29.5], [0.0, 0.0, 1.0]])
SIZE = (80, 60)


def centres(n, s):
    c = ORIGIN[0] + (np.arange(n, dtype=np.float64) + 0.5) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


def plane_volume(z0):
    _, _, z = centres(N, S_G)
    F = np.clip((z - z0) / MU, -1.0, 1.0).astype(np.float32)
    return F, np.ones_like(F, np.uint8)


def sphere_volume(c, r):
    x, y, z = centres(N, S_G)
    dist = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    F = np.clip((dist - r) / MU, -1.0, 1.0).astype(np.float32)
    return F, np.ones_like(F, np.uint8)


def coded_colours(nc):
    return (np.arange(nc ** 3, dtype=np.uint32).reshape(nc, nc, nc) & 0xFFFFFF) | (7 << 24)


def look_down(cx, cy, cz):
    T = np.eye(4)
    T[:3, :3] = np.diag([1.0, -1.0, -1.0])  # camera z (forward) = world -z
    T[:3, 3] = [cx, cy, cz]
    return T


def rays(T):
    """Unit world directions of every pixel (binary64)."""
    xs, ys = np.meshgrid(np.arange(SIZE[0], dtype=np.float64), np.arange(SIZE[1], dtype=np.float64))
    dc = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(K).T
    d = dc @ np.asarray(T, np.float64)[:3, :3].T
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_plane_from_above_closed_form(oracle_lib):
    z0 = -0.1
    F, W = plane_volume(z0)
    C = coded_colours(2 * N)
    T = look_down(0.03, -0.02, 0.35)
    r = oracle.raycast(F, W, C, S_G, S_G / 2, ORIGIN, K, T, SIZE, near=0.05, far=2.0, mu=MU)
    assert r["hits"] == SIZE[0] * SIZE[1]
    d = rays(T)
    t_exact = (T[2, 3] - z0) / -d[..., 2]
    np.testing.assert_allclose(r["range"], t_exact, rtol=0, atol=2e-5)
    np.testing.assert_allclose(r["vertex"][..., 2], z0, rtol=0, atol=2e-5)
    v_exact = T[:3, 3] + t_exact[..., None] * d
    np.testing.assert_allclose(r["vertex"], v_exact, rtol=0, atol=3e-5)
    # the TSDF gradient of a horizontal plane seen from above points up
    np.testing.assert_allclose(r["normal"], np.broadcast_to([0.0, 0.0, 1.0], r["normal"].shape), atol=1e-6)
    # colour: the code of the colour voxel holding the vertex (away from voxel faces)
    g = (r["vertex"].astype(np.float64) - np.asarray(ORIGIN)) / (S_G / 2)
    k = np.floor(g).astype(np.int64)
    clear = np.all(np.abs(g - np.round(g)) > 1e-3, axis=-1)
    assert clear.mean() > 0.9
    code = ((k[..., 2] * 2 * N + k[..., 1]) * 2 * N + k[..., 0]) & 0xFFFFFF | (7 << 24)
    np.testing.assert_array_equal(r["rgbw"][clear], code[clear].astype(np.uint32))


@pytest.mark.parametrize("oblique", [False, True])
def test_sphere_hits_lie_on_the_sphere_with_radial_normals(oracle_lib, oblique):
    from paper_1602_06645_gb300 import synth
    c, rad = np.array([0.02, -0.03, -0.05]), 0.22
    F, W = sphere_volume(c, rad)
    if oblique:
        T = synth.look_at((0.33, -0.21, 0.3), c + np.array([0.03, 0.02, 0.0]))
    else:
        T = look_down(0.0, 0.0, 0.45)
    r = oracle.raycast(F, W, None, S_G, S_G, ORIGIN, K, T, SIZE, near=0.05, far=2.0, mu=MU)
    hit = r["range"] > 0
    d = rays(T)
    # closed form: the ray hits the sphere iff the discriminant is positive
    o = T[:3, 3]
    b = (d * (o - c)).sum(-1)
    disc = b * b - ((o - c) ** 2).sum() + rad * rad
    sure_hit, sure_miss = disc > 0.02 * rad * rad, disc < -0.02 * rad * rad
    assert np.all(hit[sure_hit]) and not np.any(hit[sure_miss]) and sure_hit.sum() > 1000
    t_exact = -b - np.sqrt(np.maximum(disc, 0))
    np.testing.assert_allclose(r["range"][sure_hit], t_exact[sure_hit], atol=0.15 * S_G)
    v = r["vertex"][hit].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(v - c, axis=-1), rad, atol=0.15 * S_G)
    n = r["normal"][hit].astype(np.float64)
    radial = (v - c) / np.linalg.norm(v - c, axis=-1, keepdims=True)
    cosang = (n * radial).sum(-1)
    assert np.all(cosang > math.cos(math.radians(4.0)))
    np.testing.assert_allclose(np.linalg.norm(n, axis=-1), 1.0, atol=1e-6)


def test_no_hits_without_observations_looking_away_or_from_inside(oracle_lib):
    F, W = sphere_volume(np.zeros(3), 0.2)
    T = look_down(0.0, 0.0, 0.45)
    r = oracle.raycast(F, np.zeros_like(W), None, S_G, S_G, ORIGIN, K, T, SIZE, near=0.05, far=2.0, mu=MU)
    assert r["hits"] == 0 and not r["range"].any() and not r["vertex"].any()
    up = T.copy()
    up[:3, :3] = np.diag([1.0, 1.0, 1.0])  # camera forward = world +z, away from the sphere
    assert oracle.raycast(F, W, None, S_G, S_G, ORIGIN, K, up, SIZE, near=0.05, far=2.0, mu=MU)["hits"] == 0
    inside = look_down(0.0, 0.0, 0.0)  # at the centre: rays only leave the solid (- to +)
    assert oracle.raycast(F, W, None, S_G, S_G, ORIGIN, K, inside, SIZE, near=0.0, far=2.0, mu=MU)["hits"] == 0


def test_first_surface_along_the_ray_is_taken(oracle_lib):
    """Two horizontal planes: the union's distance field is the nearer one from
    above; every ray stops at the upper plane."""
    _, _, z = centres(N, S_G)
    up, low = 0.05, -0.2
    sd = np.where(z > (up + low) / 2, z - up, low - z)
    F = np.clip(sd / MU, -1.0, 1.0).astype(np.float32)
    T = look_down(0.0, 0.0, 0.4)
    r = oracle.raycast(F, np.ones_like(F, np.uint8), None, S_G, S_G, ORIGIN, K, T, SIZE, near=0.05, far=2.0,
                       mu=MU)
    assert r["hits"] == SIZE[0] * SIZE[1]
    np.testing.assert_allclose(r["vertex"][..., 2], up, atol=2e-5)
