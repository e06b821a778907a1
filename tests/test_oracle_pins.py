"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test computes its expectation by a route independent of the oracle's
code: closed-form depths along pixel rays, counting invariants, integer
identities of the colour average, pixel-coded images that reveal which HD
pixel a voxel sampled, and an occluder that only the Eq. 7 sigma gate can
reject.  A plausible slip in the oracle (a transposed pose, a swapped u/v, a
dropped truncation, a wrong sign, nearest in place of bilinear) fails at
least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from fp64_model import EPS_M, EPS_PX, Model, _round_tie


# ----------------------------------------------------------------- helpers
def K_of(f, W, H):
    return np.array([[f, 0, (W - 1) / 2.0], [0, f, (H - 1) / 2.0], [0, 0, 1]], np.float32)


def rot(axis, deg):
    a = np.asarray(axis, np.float64)
    a /= np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    th = math.radians(deg)
    return np.eye(3) + math.sin(th) * k + (1 - math.cos(th)) * k @ k


def pose(axis=(0.3, -0.5, 0.8), deg=20.0, t=(0.1, -0.2, 0.3)):
    T = np.eye(4)
    T[:3, :3] = rot(axis, deg)
    T[:3, 3] = t
    return T.astype(np.float32)


def plane_Z(K, iu, iv, z0, a=0.0, b=0.0):
    """Camera-frame Z where the ray through pixel (iu, iv) meets the plane
    Z = z0 + a X + b Y (closed form: X = Z rx, Y = Z ry on that ray)."""
    Ki = np.linalg.inv(np.asarray(K, np.float64))
    rx = Ki[0, 0] * iu + Ki[0, 1] * iv + Ki[0, 2]
    ry = Ki[1, 0] * iu + Ki[1, 1] * iv + Ki[1, 2]
    rz = Ki[2, 0] * iu + Ki[2, 1] * iv + Ki[2, 2]
    rx, ry = rx / rz, ry / rz
    return z0 / (1.0 - a * rx - b * ry)


def plane_depth_image(K, W, H, z0, a=0.0, b=0.0):
    iv, iu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    Z = plane_Z(K, iu, iv, z0, a, b)
    return np.floor(Z * 1000.0 + 0.5).astype(np.uint16)


def centres_world(dims, s, origin):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (origin[0] + (x + 0.5) * s, origin[1] + (y + 0.5) * s, origin[2] + (z + 0.5) * s)


def world_to_cam(T, X, Y, Z):
    T = np.asarray(T, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    d = (X - t[0], Y - t[1], Z - t[2])
    return tuple(R[0, r] * d[0] + R[1, r] * d[1] + R[2, r] * d[2] for r in range(3))


def box_in_front(T, dims, s, dist):
    """Origin of a volume of `dims` voxels of size s centred `dist` in front of camera T."""
    c = np.asarray(T, np.float64) @ np.array([0, 0, dist, 1.0])
    return tuple(float(np.float32(c[a] - dims[a] * s / 2.0)) for a in range(3))


def expected_plane_tsdf(dims, s, origin, T, K, W, H, mu, z0, a=0.0, b=0.0):
    """Closed-form single-frame TSDF of the plane: per voxel the pixel it
    projects to (nearest), the mm-quantised analytic depth at that pixel,
    sdf = D/1000 - Z, update iff sdf >= -mu, F = min(1, sdf/mu).  Also returns
    the near-tie mask."""
    X, Y, Z = world_to_cam(T, *centres_world(dims, s, origin))
    K = np.asarray(K, np.float64)
    u = K[0, 0] * X / Z + K[0, 2]
    v = K[1, 1] * Y / Z + K[1, 2]
    fu, fv = np.floor(u + 0.5), np.floor(v + 0.5)
    inside = (Z > 0) & (fu >= 0) & (fu <= W - 1) & (fv >= 0) & (fv <= H - 1)
    D = np.floor(plane_Z(K, fu, fv, z0, a, b) * 1000.0 + 0.5)
    sdf = D * 1e-3 - Z
    upd = inside & (sdf >= -mu)
    F = np.where(upd, np.minimum(1.0, sdf / mu), 0.0)
    tie = _round_tie(u) | _round_tie(v) | (np.abs(sdf + mu) < EPS_M)
    return upd, F, tie, sdf


# ------------------------------------------------------ geometry (TSDF) pins
GEO = dict(dims=(24, 20, 16), s=0.02, mu=0.05)
IMG = (80, 60)


@pytest.mark.parametrize("a,b", [(0.0, 0.0), (0.2, -0.1)])
def test_plane_tsdf_closed_form(oracle_lib, a, b):
    """One frame of a (tilted) plane seen from an arbitrary pose: every voxel's
    TSDF and weight equal the closed form.  Pins Eq. 5 (pose direction),
    Eq. 6 (projection, u from X, v from Y), depth units, sdf sign, truncation."""
    W, H = IMG
    K = K_of(70.0, W, H)
    T = pose()
    dims, s, mu = GEO["dims"], GEO["s"], GEO["mu"]
    origin = box_in_front(T, dims, s, 0.9)
    depth = plane_depth_image(K, W, H, 0.9, a, b)
    o = oracle.Oracle(dims, dims, s, mu, 10, origin=origin)
    n = o.integrate_geometry(depth, K, T)
    upd, F, tie, sdf = expected_plane_tsdf(dims, s, origin, T, K, W, H, mu, 0.9, a, b)
    ok = ~tie
    assert n == int(o.W.astype(bool).sum())
    np.testing.assert_array_equal(o.W[ok], upd[ok].astype(np.uint8))
    np.testing.assert_allclose(o.F[ok], F[ok].astype(np.float32), atol=1e-5, rtol=0)
    # the case covers free space, the band and the hidden region
    assert (upd & ok & (sdf > mu)).sum() > 100
    assert (upd & ok & (np.abs(sdf) < mu)).sum() > 100
    inside_hidden = ok & ~upd & (sdf < -mu) & np.isfinite(sdf)
    assert inside_hidden.sum() > 100


def sphere_Z(K, iu, iv, c, r):
    """Camera-frame Z of the first point where the ray through pixel (iu, iv)
    meets the sphere |P - c| = r (closed form: P = Z d with d = K^-1 (iu, iv, 1)
    scaled to d_z = 1, so Z^2 |d|^2 - 2 Z d.c + |c|^2 - r^2 = 0, smaller root);
    NaN where the ray misses or the sphere is behind the camera."""
    Ki = np.linalg.inv(np.asarray(K, np.float64))
    d = [Ki[i, 0] * iu + Ki[i, 1] * iv + Ki[i, 2] for i in range(3)]
    d = [d[0] / d[2], d[1] / d[2], np.ones_like(d[2])]
    dd = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
    dc = d[0] * c[0] + d[1] * c[1] + d[2] * c[2]
    disc = dc * dc - dd * (c[0] ** 2 + c[1] ** 2 + c[2] ** 2 - r * r)
    with np.errstate(invalid="ignore"):
        Z = (dc - np.sqrt(disc)) / dd
    return np.where((disc >= 0) & (Z > 0), Z, np.nan)


def expected_sphere_tsdf(dims, s, origin, T, K, W, H, mu, c, r):
    """Closed-form single-frame TSDF of a sphere (centre c, radius r in the
    camera frame): per voxel its nearest pixel, the mm-quantised depth of the
    sphere along that pixel's ray (no depth where the ray misses),
    sdf = D/1000 - Z, updated iff D > 0 and sdf >= -mu, F = min(1, sdf/mu).
    Also returns the near-tie mask."""
    X, Y, Z = world_to_cam(T, *centres_world(dims, s, origin))
    K = np.asarray(K, np.float64)
    u = K[0, 0] * X / Z + K[0, 2]
    v = K[1, 1] * Y / Z + K[1, 2]
    fu, fv = np.floor(u + 0.5), np.floor(v + 0.5)
    inside = (Z > 0) & (fu >= 0) & (fu <= W - 1) & (fv >= 0) & (fv <= H - 1)
    Zs = sphere_Z(K, fu, fv, c, r)
    hit = np.isfinite(Zs)
    D = np.where(hit, np.floor(np.nan_to_num(Zs) * 1000.0 + 0.5), 0.0)
    sdf = D * 1e-3 - Z
    upd = inside & (D > 0) & (sdf >= -mu)
    F = np.where(upd, np.minimum(1.0, sdf / mu), 0.0)
    tie = _round_tie(u) | _round_tie(v) | (np.abs(sdf + mu) < EPS_M)
    return upd, F, tie, sdf


def sphere_depth_image(K, W, H, c, r):
    iv, iu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    Z = sphere_Z(K, iu, iv, c, r)
    return np.where(np.isfinite(Z), np.floor(np.nan_to_num(Z) * 1000.0 + 0.5), 0).astype(np.uint16)


SPHERE = dict(c=(0.04, -0.03, 0.8), r=0.15)


def test_sphere_tsdf_closed_form(oracle_lib):
    """One frame of a sphere: every voxel's TSDF and weight equal the
    projective closed form through its rounded pixel ray, including voxels
    whose ray misses the sphere (no depth, not updated) and the silhouette."""
    W, H = IMG
    K = K_of(70.0, W, H)
    T = pose(deg=35.0)
    dims, s, mu = GEO["dims"], GEO["s"], GEO["mu"]
    origin = box_in_front(T, dims, s, 0.8)
    depth = sphere_depth_image(K, W, H, SPHERE["c"], SPHERE["r"])
    assert (depth == 0).sum() > 100 and (depth > 0).sum() > 100
    o = oracle.Oracle(dims, dims, s, mu, 10, origin=origin)
    n = o.integrate_geometry(depth, K, T)
    upd, F, tie, sdf = expected_sphere_tsdf(dims, s, origin, T, K, W, H, mu, SPHERE["c"], SPHERE["r"])
    ok = ~tie
    assert n == int(o.W.astype(bool).sum())
    np.testing.assert_array_equal(o.W[ok], upd[ok].astype(np.uint8))
    np.testing.assert_allclose(o.F[ok], F[ok].astype(np.float32), atol=1e-5, rtol=0)
    assert (upd & ok & (np.abs(sdf) < mu)).sum() > 100  # the band around the curved surface
    assert (upd & ok & (sdf > mu)).sum() > 100
    assert (ok & ~upd & (sdf < -mu) & (F == 0)).sum() > 10  # hidden inside the sphere


def test_sphere_tsdf_two_views_average(oracle_lib):
    """Two frames of the same sphere from two camera poses: voxels updated in
    both hold the mean of the two closed forms, in one the single value; the
    weight counts the frames."""
    W, H = IMG
    K = K_of(70.0, W, H)
    dims, s, mu = GEO["dims"], GEO["s"], GEO["mu"]
    T1 = pose(deg=10.0, t=(0.0, 0.0, 0.0))
    c_world = np.asarray(T1, np.float64) @ np.array([*SPHERE["c"], 1.0])
    T2 = np.asarray(T1, np.float64).copy()
    R2 = rot((0.0, 1.0, 0.0), 12.0)
    # second camera: rotated about the sphere centre by 12 degrees
    T2[:3, :3] = R2 @ T1[:3, :3]
    T2[:3, 3] = c_world[:3] + R2 @ (T1[:3, 3] - c_world[:3])
    T2 = T2.astype(np.float32)
    origin = box_in_front(T1, dims, s, 0.8)
    o = oracle.Oracle(dims, dims, s, mu, 10, origin=origin)
    ups, Fs, ties = [], [], []
    for Tk in (T1, T2):
        Tk64 = np.asarray(Tk, np.float64)
        c_cam = Tk64[:3, :3].T @ (c_world[:3] - Tk64[:3, 3])
        depth = sphere_depth_image(K, W, H, c_cam, SPHERE["r"])
        o.integrate_geometry(depth, K, Tk)
        u, F, tie, _ = expected_sphere_tsdf(dims, s, origin, Tk, K, W, H, mu, c_cam, SPHERE["r"])
        ups.append(u)
        Fs.append(F)
        ties.append(tie)
    ok = ~(ties[0] | ties[1])
    both = ups[0] & ups[1]
    wexp = ups[0].astype(np.uint8) + ups[1].astype(np.uint8)
    np.testing.assert_array_equal(o.W[ok], wexp[ok])
    Fexp = np.where(both, 0.5 * (Fs[0] + Fs[1]), Fs[0] + Fs[1])
    np.testing.assert_allclose(o.F[ok], Fexp[ok].astype(np.float32), atol=1e-5, rtol=0)
    assert (both & ok).sum() > 500 and (ok & (wexp == 1)).sum() > 50


@pytest.mark.parametrize("max_w", [1, 4, 255])
def test_weight_counts_observing_frames(oracle_lib, max_w):
    """n identical frames: weight = min(n, max_weight) where observed, 0 elsewhere;
    the TSDF of identical samples stays that sample."""
    W, H = IMG
    K = K_of(70.0, W, H)
    T = pose()
    dims, s, mu = GEO["dims"], GEO["s"], GEO["mu"]
    origin = box_in_front(T, dims, s, 0.9)
    depth = plane_depth_image(K, W, H, 0.9, 0.2, -0.1)
    o = oracle.Oracle(dims, dims, s, mu, max_w, origin=origin)
    n = 6
    for _ in range(n):
        o.integrate_geometry(depth, K, T)
    upd, F, tie, _ = expected_plane_tsdf(dims, s, origin, T, K, W, H, mu, 0.9, 0.2, -0.1)
    ok = ~tie
    np.testing.assert_array_equal(o.W[ok], np.where(upd[ok], min(n, max_w), 0).astype(np.uint8))
    np.testing.assert_allclose(o.F[ok], F[ok], atol=1e-5, rtol=0)


@pytest.mark.parametrize("max_w", [1, 2, 64])
def test_running_average_and_cap(oracle_lib, max_w):
    """Three frames of fronto-parallel planes at different depths: F is the
    running weighted average (F w + t)/(w + 1), and averaging continues with
    w = max_weight once the cap is reached."""
    W, H = IMG
    K = K_of(70.0, W, H)
    T = np.eye(4, dtype=np.float32)
    dims, s, mu = GEO["dims"], GEO["s"], GEO["mu"]
    origin = box_in_front(T, dims, s, 0.9)
    zs = [0.90, 0.93, 0.87]
    o = oracle.Oracle(dims, dims, s, mu, max_w, origin=origin)
    Fe = np.zeros(dims[::-1])
    We = np.zeros(dims[::-1])
    tie = np.zeros(dims[::-1], bool)
    for z0 in zs:
        o.integrate_geometry(plane_depth_image(K, W, H, z0), K, T)
        upd, t, ti, _ = expected_plane_tsdf(dims, s, origin, T, K, W, H, mu, z0)
        Fe = np.where(upd, (Fe * We + t) / (We + 1), Fe)
        We = np.where(upd, np.minimum(We + 1, max_w), We)
        tie |= ti
    ok = ~tie
    np.testing.assert_array_equal(o.W[ok], We[ok].astype(np.uint8))
    np.testing.assert_allclose(o.F[ok], Fe[ok], atol=1e-5, rtol=0)
    assert (ok & (We == min(3, max_w))).sum() > 200


# ----------------------------------------------------------- colour pins
def colour_setup(ratio=2, z0=0.9, pose_T=None, s=0.03, gdims=(20, 16, 12)):
    W, H = IMG
    Kd = K_of(70.0, W, H)
    T = pose() if pose_T is None else pose_T
    cdims = tuple(d * ratio for d in gdims)
    origin = box_in_front(T, gdims, s, z0)
    depth = plane_depth_image(Kd, W, H, z0)
    Tdr = np.eye(4)
    Tdr[:3, :3] = rot((0, 1, 0), 3.0)
    Tdr[:3, 3] = (-0.05, 0.0, 0.0)
    return W, H, Kd, T, gdims, cdims, s, origin, depth, Tdr.astype(np.float32)


def pixel_code_image(W, H):
    iv, iu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = np.zeros((H, W, 3), np.uint8)
    img[..., 0] = iu % 256
    img[..., 1] = iv % 256
    img[..., 2] = (iu // 256) + 16 * (iv // 256)
    return img


def test_constant_colour_gives_constant_volume(oracle_lib):
    """A constant HD image leaves every updated colour voxel at exactly that
    colour: (c (w+1) + floor((w+1)/2)) div (w+1) = c for all w."""
    from paper_1602_06645_gb300 import synth
    seq = synth.sequence_small(n_frames=3, dims_geo=32)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    col = np.array([77, 140, 201], np.uint8)
    for f in range(3):
        d, _ = seq.frame(f)
        rgb = np.broadcast_to(col, (seq.rgb_size[1], seq.rgb_size[0], 3))
        o.integrate(d, rgb, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    w = o.colour_weight
    assert (w > 0).sum() > 1000 and (w > 1).sum() > 100
    assert np.all(o.colour_rgb[w > 0] == col)
    assert np.all(o.colour_rgb[w == 0] == 0)


@pytest.mark.parametrize("ratio", [1, 2, 3])
def test_colour_samples_the_calibrated_hd_pixel(oracle_lib, ratio):
    """Pixel-coded HD image: each updated colour voxel holds the code of the
    HD pixel that Eq. 3-4 map it to (through R_calib, t_calib and K_hd), at
    every asymmetry ratio.  The set of updated voxels equals the binary64
    evaluation of the Eq. 6/7 and band gates away from near ties."""
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(ratio)
    cW, cH = 128, 96
    Kr = K_of(90.0, cW, cH)
    rgb = pixel_code_image(cW, cH)
    mu = 0.08
    o = oracle.Oracle(gd, cd, s, mu, 64, origin=origin)
    o.integrate(depth, rgb, Kd, Kr, T, Tdr)
    m = Model(gd, cd, s, o.p.s_c, origin, mu, 64, 0.020, o.p.band)
    m.integrate(depth, rgb, Kd, Kr, T, Tdr)
    ok = ~m.tie_c
    got = o.colour_weight > 0
    np.testing.assert_array_equal(got[ok], m.CW[ok] > 0)
    # at ratio 1 every colour centre sits on a geometry centre, so the
    # trilinear cell is always a near tie there; the decode below still runs
    assert got.sum() > 50 and (ratio == 1 or (got & ok).sum() > 50)
    # decode the sampled pixel and compare with the binary64 HD projection
    Xc, Yc, Zc = world_to_cam(T, *centres_world(cd, o.p.s_c, origin))
    Td = np.asarray(Tdr, np.float64)
    P = [Td[r, 0] * Xc + Td[r, 1] * Yc + Td[r, 2] * Zc + Td[r, 3] for r in range(3)]
    uh = 90.0 * P[0] / P[2] + (cW - 1) / 2.0
    vh = 90.0 * P[1] / P[2] + (cH - 1) / 2.0
    sel = got & ~(_round_tie(uh) | _round_tie(vh))
    rgbv = o.colour_rgb
    code_u = rgbv[..., 0].astype(int) + 256 * (rgbv[..., 2].astype(int) % 16)
    code_v = rgbv[..., 1].astype(int) + 256 * (rgbv[..., 2].astype(int) // 16)
    np.testing.assert_array_equal(code_u[sel], np.floor(uh[sel] + 0.5).astype(int))
    np.testing.assert_array_equal(code_v[sel], np.floor(vh[sel] + 0.5).astype(int))


def test_band_gate_selects_near_surface_voxels(oracle_lib):
    """Fronto-parallel plane seen head on: the trilinear TSDF is linear in Z,
    so a colour voxel is updated only within band * mu of the surface (and
    with a band of 10, i.e. disabled, everywhere the Eq. 7 gate passes)."""
    T = np.eye(4, dtype=np.float32)
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2, pose_T=T)
    Kr = K_of(90.0, 128, 96)
    rgb = pixel_code_image(128, 96)
    mu = 0.08
    for band, sigma in [(None, 0.02), (10.0, 0.05)]:
        o = oracle.Oracle(gd, cd, s, mu, 64, origin=origin, band=band, sigma=sigma)
        o.integrate(depth, rgb, Kd, Kr, T, Tdr)
        m = Model(gd, cd, s, o.p.s_c, origin, mu, 64, sigma, o.p.band)
        m.integrate(depth, rgb, Kd, Kr, T, Tdr)
        ok = ~m.tie_c
        got = o.colour_weight > 0
        np.testing.assert_array_equal(got[ok], m.CW[ok] > 0)
        Xc, Yc, Zc = centres_world(cd, o.p.s_c, origin)
        dz = np.abs(Zc - 0.9)
        if band is None:
            # within one colour voxel (band = s_c/mu) of the surface, plus the
            # depth quantisation of half a millimetre
            assert got.any() and dz[got].max() <= o.p.band * mu + 0.6e-3
        else:
            assert dz[got].max() > 2 * o.p.s_c


def test_sigma_gate_rejects_occluded_voxels(oracle_lib):
    """Eq. 7: frame 1 sees a plane in colour A; frame 2 sees the same plane in
    colour B except behind a square occluder 0.3 m in front of it.  Voxels on
    the plane behind the occluder keep colour A and weight 1 (the depth pixel
    they project to lies on the occluder, far beyond sigma = 20 mm); the others
    average to (A + B + 1) div 2 with weight 2.  With sigma disabled the
    occluded voxels would take the occluder's colour."""
    T = np.eye(4, dtype=np.float32)
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2, pose_T=T)
    Tdr = np.eye(4, dtype=np.float32)  # HD camera = depth camera, so the occluder hides the same pixels
    cW, cH = W, H
    Kr = Kd.copy()
    A = np.array([200, 10, 10], np.uint8)
    B = np.array([10, 200, 10], np.uint8)
    occ = np.array([5, 5, 250], np.uint8)
    rgb1 = np.broadcast_to(A, (cH, cW, 3)).copy()
    depth2 = depth.copy()
    rgb2 = np.broadcast_to(B, (cH, cW, 3)).copy()
    sq = (slice(20, 40), slice(30, 50))
    depth2[sq] = 600
    rgb2[sq] = occ
    res = {}
    for sigma in (0.020, 10.0):
        o = oracle.Oracle(gd, cd, s, 0.08, 64, origin=origin, sigma=sigma)
        o.integrate(depth, rgb1, Kd, Kr, T, Tdr)
        o.integrate(depth2, rgb2, Kd, Kr, T, Tdr)
        res[sigma] = o
    o = res[0.020]
    Xc, Yc, Zc = centres_world(cd, o.p.s_c, origin)
    u = 70.0 * Xc / Zc + (W - 1) / 2.0
    v = 70.0 * Yc / Zc + (H - 1) / 2.0
    fu, fv = np.floor(u + 0.5), np.floor(v + 0.5)
    behind = (fu >= 31) & (fu <= 48) & (fv >= 21) & (fv <= 38)
    clear = ((fu <= 27) | (fu >= 52)) & (fv >= 0) & (fv <= H - 1) & (fu >= 0) & (fu <= W - 1)
    w = o.colour_weight
    hit_b = behind & (w > 0)
    hit_c = clear & (w > 0)
    assert hit_b.sum() > 20 and hit_c.sum() > 20
    assert np.all(w[hit_b] == 1) and np.all(o.colour_rgb[hit_b] == A)
    assert np.all(w[hit_c] == 2) and np.all(o.colour_rgb[hit_c] == (A.astype(int) + B + 1) // 2)
    # without the sigma gate the hidden voxels take the occluder's colour
    o2 = res[10.0]
    w2 = o2.colour_weight
    assert np.all(w2[hit_b] == 2)
    assert np.all(o2.colour_rgb[hit_b] == (A.astype(int) + occ + 1) // 2)


def test_sigma_is_in_metres(oracle_lib):
    """The gate compares |P_vc - P_vd| with sigma in metres: a plane with
    band disabled updates voxels up to sigma away from the measured depth."""
    T = np.eye(4, dtype=np.float32)
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2, pose_T=T, s=0.01, gdims=(20, 16, 20))
    Kr = K_of(90.0, 128, 96)
    rgb = pixel_code_image(128, 96)
    for sigma in (0.012, 0.03):
        o = oracle.Oracle(gd, cd, 0.01, 0.2, 64, origin=origin, band=10.0, sigma=sigma)
        o.integrate(depth, rgb, Kd, Kr, T, Tdr)
        Xc, Yc, Zc = centres_world(cd, o.p.s_c, origin)
        got = o.colour_weight > 0
        dz = np.abs(Zc - 0.9)
        assert dz[got].max() <= sigma + 1e-3
        assert dz[got].max() >= sigma - o.p.s_c - 1e-3


def test_bilinear_sampling_of_a_linear_ramp(oracle_lib):
    """Bilinear interpolation reproduces a linear image exactly, so with
    R = 2 x and G = 2 y the sample is round_half_up(2 u_hd) and
    round_half_up(2 v_hd); nearest sampling would give 2 round(u_hd)."""
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2)
    cW, cH = 120, 100
    Kr = K_of(90.0, cW, cH)
    iv, iu = np.meshgrid(np.arange(cH), np.arange(cW), indexing="ij")
    rgb = np.stack([2 * iu, 2 * iv, np.full_like(iu, 7)], -1).astype(np.uint8)
    res = {}
    for mode in (0, 1):
        o = oracle.Oracle(gd, cd, s, 0.08, 64, origin=origin, sample_mode=mode)
        o.integrate(depth, rgb, Kd, Kr, T, Tdr)
        res[mode] = o
    o = res[1]
    Xc, Yc, Zc = world_to_cam(T, *centres_world(cd, o.p.s_c, origin))
    Td = np.asarray(Tdr, np.float64)
    P = [Td[r, 0] * Xc + Td[r, 1] * Yc + Td[r, 2] * Zc + Td[r, 3] for r in range(3)]
    uh = 90.0 * P[0] / P[2] + (cW - 1) / 2.0
    vh = 90.0 * P[1] / P[2] + (cH - 1) / 2.0
    got = o.colour_weight > 0
    frac = lambda x: np.abs(np.mod(x + 0.5, 1.0) - 0.5)
    sel = got & (frac(2 * uh + 0.5 - 0.5) > 1e-3) & (frac(2 * vh) > 1e-3)
    sel &= (np.abs(uh - np.round(uh)) > 1e-3) & (np.abs(vh - np.round(vh)) > 1e-3)
    assert sel.sum() > 50
    rgbv = o.colour_rgb.astype(int)
    np.testing.assert_array_equal(rgbv[sel, 0], np.floor(2 * uh[sel] + 0.5).astype(int))
    np.testing.assert_array_equal(rgbv[sel, 1], np.floor(2 * vh[sel] + 0.5).astype(int))
    assert np.all(rgbv[sel, 2] == 7)
    # nearest mode differs on a large share of the same voxels
    near = res[0].colour_rgb.astype(int)
    both = sel & (res[0].colour_weight > 0)
    assert (near[both, 0] != rgbv[both, 0]).mean() > 0.2


def test_colour_average_rounds_half_up(oracle_lib):
    """Three identical-geometry frames in colours A, B, C: a voxel seen by all
    three holds ((((A+B+1) div 2) * 2 + C + 1) div 3) per channel (Eq. 9 with
    W = 1, integer half-up rounding)."""
    T = np.eye(4, dtype=np.float32)
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2, pose_T=T)
    Kr = K_of(90.0, 128, 96)
    cols = [np.array(c, np.uint8) for c in ([200, 3, 100], [51, 4, 17], [0, 255, 90])]
    o = oracle.Oracle(gd, cd, s, 0.08, 64, origin=origin)
    for c in cols:
        o.integrate(depth, np.broadcast_to(c, (96, 128, 3)), Kd, Kr, T, Tdr)
    A, B, C = [c.astype(int) for c in cols]
    e2 = (A + B + 1) // 2
    e3 = (e2 * 2 + C + 1) // 3
    w = o.colour_weight
    assert (w == 3).sum() > 50
    assert np.all(o.colour_rgb[w == 3] == e3)


def test_paper_normal_weight_is_view_cosine(oracle_lib):
    """Colour mode 1 (Eq. 8-10).  A fronto-parallel plane has its normal along
    the optical axis, so W = cos(angle between the viewing ray and the axis)
    = Z / |P_vc|, stored as round(255 W).  A second identical frame in another
    colour passes the 0.8 W_pre gate, averages the colours as
    (A + B + 1) div 2, and saturates the weight by Eq. 10:
    w2 = w1 + (w1 (255 - w1) + 127) div 255.  A third identical frame passes
    the gate only where 5 w1 > 4 w2."""
    T = np.eye(4, dtype=np.float32)
    W, H, Kd, T, gd, cd, s, origin, depth, Tdr = colour_setup(2, pose_T=T, gdims=(80, 60, 8), s=0.02)
    Tdr = np.eye(4, dtype=np.float32)
    Kd = K_of(35.0, W, H)  # wide field of view: viewing angles up to ~50 degrees
    Kr = Kd.copy()
    depth = plane_depth_image(Kd, W, H, 0.9)
    A = np.array([200, 40, 0], np.uint8)
    B = np.array([0, 90, 255], np.uint8)
    o = oracle.Oracle(gd, cd, 0.02, 0.08, 64, origin=origin, colour_mode=1)
    o.integrate(depth, np.broadcast_to(A, (H, W, 3)), Kd, Kr, T, Tdr)
    Xc, Yc, Zc = centres_world(cd, o.p.s_c, origin)
    cosv = Zc / np.sqrt(Xc ** 2 + Yc ** 2 + Zc ** 2)
    wq = np.floor(255 * cosv + 0.5)
    tie = np.abs(np.mod(255 * cosv + 0.5, 1.0) - 0.5) > 0.5 - 1e-3
    w1 = o.colour_weight.astype(int)
    got = (w1 > 0) & ~tie
    assert got.sum() > 100 and wq[got].min() < 200
    np.testing.assert_array_equal(w1[got], wq[got].astype(int))
    assert np.all(o.colour_rgb[w1 > 0] == A)
    o.integrate(depth, np.broadcast_to(B, (H, W, 3)), Kd, Kr, T, Tdr)
    w2 = o.colour_weight.astype(int)
    np.testing.assert_array_equal(w2[got], w1[got] + (w1[got] * (255 - w1[got]) + 127) // 255)
    assert np.all(o.colour_rgb[got] == (A.astype(int) + B + 1) // 2)
    o.integrate(depth, np.broadcast_to(A, (H, W, 3)), Kd, Kr, T, Tdr)
    w3 = o.colour_weight.astype(int)
    passes = 5 * w1 > 4 * w2
    assert (got & passes).sum() > 20 and (got & ~passes).sum() > 20
    np.testing.assert_array_equal(w3[got & ~passes], w2[got & ~passes])
    gp = got & passes
    np.testing.assert_array_equal(w3[gp], w2[gp] + (w1[gp] * (255 - w2[gp]) + 127) // 255)


# ------------------------------------------------------ frame constants pin
def test_frame_constants_invert_the_pose(oracle_lib):
    """(R_n, t_n) of Eq. 5 is the inverse of T_world_depth, and K_c^-1 the
    matrix inverse of K_c, each rounded once to binary32."""
    T = pose((1.0, 2.0, -0.5), 37.0, (0.4, -1.1, 2.3))
    K = np.array([[525, 0.3, 319.5], [0, 530, 239.5], [0, 0, 1]], np.float32)
    o = oracle.Oracle((8, 8, 8), (8, 8, 8), 0.1, 0.3, 10)
    R, t, Kdi = o.frame_constants(K, K, T, np.eye(4, dtype=np.float32))
    Ti = np.linalg.inv(T.astype(np.float64))
    np.testing.assert_array_equal(R, T[:3, :3].T)
    np.testing.assert_allclose(t, Ti[:3, 3], rtol=0, atol=2e-7 * 3)
    np.testing.assert_allclose(Kdi, np.linalg.inv(K.astype(np.float64)), rtol=1e-7, atol=1e-9)


# ---------------------------------------------------- brute force, tiny sizes
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("sample_mode", [0, 1])
def test_brute_force_tiny_volumes_match_binary64(oracle_lib, seed, sample_mode):
    """8^3 geometry / 16^3 colour, random poses looking at the volume, random
    depth and RGB images, four frames: weights and colours equal the binary64
    evaluation exactly and the TSDF within 1e-5, away from near ties."""
    rng = np.random.default_rng(1000 + seed)
    W, H = 32, 24
    Kd = K_of(40.0, W, H)
    cW, cH = 48, 36
    Kr = K_of(60.0, cW, cH)
    gd, cd, s = (8, 8, 8), (16, 16, 16), 0.05
    mu = 0.1
    origin = (-0.2, -0.2, -0.2)
    o = oracle.Oracle(gd, cd, s, mu, 3, origin=origin, band=0.3, sample_mode=sample_mode, sigma=0.04)
    m = Model(gd, cd, s, o.p.s_c, origin, mu, 3, 0.04, 0.3, sample_mode=sample_mode)
    Tdr = np.eye(4)
    Tdr[:3, :3] = rot(rng.normal(size=3), 2.0)
    Tdr[:3, 3] = (-0.03, 0.004, 0.001)
    Tdr = Tdr.astype(np.float32)
    for f in range(4):
        az, el = rng.uniform(0, 2 * np.pi), rng.uniform(-0.6, 0.6)
        dist = rng.uniform(0.5, 0.8)
        pos = dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        from paper_1602_06645_gb300.synth import look_at
        T = look_at(pos, rng.normal(size=3) * 0.03).astype(np.float32)
        base = plane_depth_image(Kd, W, H, dist + rng.uniform(-0.05, 0.05), rng.uniform(-0.3, 0.3),
                                 rng.uniform(-0.3, 0.3)).astype(np.int64)
        depth = np.clip(base + rng.integers(-15, 16, size=base.shape), 0, 65535).astype(np.uint16)
        depth[rng.random(depth.shape) < 0.05] = 0
        rgb = rng.integers(0, 256, size=(cH, cW, 3), dtype=np.uint8)
        o.integrate(depth, rgb, Kd, Kr, T, Tdr)
        m.integrate(depth, rgb, Kd, Kr, T, Tdr)
    okg = ~m.tie_g
    okc = ~m.tie_c
    assert okg.mean() > 0.9 and okc.mean() > 0.8
    np.testing.assert_array_equal(o.W[okg], m.W[okg])
    np.testing.assert_allclose(o.F[okg], m.F[okg], atol=1e-5, rtol=0)
    np.testing.assert_array_equal(o.colour_weight[okc], m.CW[okc])
    np.testing.assert_array_equal(o.colour_rgb[okc], m.C[okc])
    assert (o.W > 0).sum() > 50
    assert (o.colour_weight > 0).sum() > 20


@pytest.mark.parametrize("colour_mode", [0, 1])
def test_sampled_replay_equals_the_dense_oracle(oracle_lib, colour_mode):
    """The sampled replay used for full-size parity applies the same per-voxel
    updates as the dense oracle: on samples chosen from the inputs (tests/
    samples.py) it gives the dense oracle's values exactly, and the geometry
    sample holds every corner the colour band gate reads."""
    from paper_1602_06645_gb300 import synth
    from samples import scan_samples
    seq = synth.sequence_small(n_frames=4, dims_geo=48, ratio=2)
    geo, col = scan_samples(seq, range(4), n_col=3000, n_geo=4000, seed=5)
    kw = dict(colour_mode=colour_mode)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **kw)
    s = oracle.SparseOracle(geo, col, seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **kw)
    for f in range(4):
        d, c = seq.frame(f)
        o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        assert s.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb) == 0
    gi, ci = s.geo_index.astype(np.int64), s.col_index.astype(np.int64)
    np.testing.assert_array_equal(o.F.reshape(-1)[gi].view(np.uint32), s.F.view(np.uint32))
    np.testing.assert_array_equal(o.W.reshape(-1)[gi], s.W)
    np.testing.assert_array_equal(o.C.reshape(-1)[ci], s.C)
    # the samples exercise the gates: most colour samples were coloured, some were not
    w = s.C >> 24
    assert 0.15 < (w > 0).mean() < 0.99 and (s.W > 0).mean() > 0.2 and (s.W == 0).any()
