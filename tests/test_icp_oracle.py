"""Pins of the camera-tracking oracle (oracle/icp.c; Section III: a vertex /
normal map pyramid of the input depth map and ICP against the surface
prediction ray-traced from the geometry volume).

Each expectation comes from outside the oracle's code: block means worked
out by hand, a plane's normals in closed form, the normal equations evaluated
independently in binary64 numpy, the rank a single plane leaves to
point-to-plane ICP, and the true poses of a synthetic sequence, which the
tracker must recover from the previous frame's pose.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1602_06645_gb300 import synth


def K_of(f, W, H):
    return np.array([[f, 0, (W - 1) / 2.0], [0, f, (H - 1) / 2.0], [0, 0, 1]], np.float32)


def test_pyramid_block_means_keep_depth_edges_apart(oracle_lib):
    D = np.array([[1000, 1010, 2000, 0],
                  [1020, 1025, 2000, 2100],
                  [0, 0, 3000, 3040],
                  [0, 500, 3020, 2980]], np.uint16)
    lv = oracle.icp_pyramid(D, 2)
    np.testing.assert_array_equal(lv[0], (D * np.float32(0.001)).astype(np.float32) * (D > 0))
    # blocks in the order (0,0), (1,0), (0,1), (1,1); depths more than 3 cm
    # from the block's first valid depth (2.1 m, 3.04 m) are left out
    want = np.array([[np.mean([1.0, 1.01, 1.02, 1.025]), 2.0],
                     [0.5, np.mean([3.0, 3.02, 2.98])]])
    np.testing.assert_allclose(lv[1], want, rtol=0, atol=1e-6)  # a few binary32 roundings
    K1 = oracle.icp_level_K(K_of(525.0, 640, 480), 1)
    np.testing.assert_allclose([K1[0, 0], K1[0, 2], K1[1, 2]], [262.5, (319.5 + 0.5) / 2 - 0.5, (239.5 + 0.5) / 2 - 0.5])


def test_plane_maps(oracle_lib):
    """Fronto-parallel plane: vertices at its depth, normals exactly (0, 0, -1)
    (toward the camera); a tilted plane Z = z0 + a X: normals along (a, 0, -1)."""
    W, H = 64, 48
    K = K_of(60.0, W, H)
    d = np.full((H, W), 0.75, np.float32)
    V, N = oracle.icp_maps(d, K)
    np.testing.assert_array_equal(V[..., 2], d)
    inner = N[:-1, :-1]
    np.testing.assert_array_equal(inner, np.broadcast_to([0.0, 0.0, -1.0], inner.shape))
    assert np.all(N[-1] == 0) and np.all(N[:, -1] == 0)
    a = 0.3
    u = np.arange(W, dtype=np.float64)
    rx = (u - K[0, 2]) / K[0, 0]
    Z = 0.75 / (1 - a * rx)  # Z = 0.75 + a X on the ray X = Z rx
    d = np.broadcast_to(Z, (H, W)).astype(np.float32)
    _, N = oracle.icp_maps(d, K)
    n = np.array([a, 0.0, -1.0]) / math.hypot(a, 1.0)
    np.testing.assert_allclose(N[:-1, :-1].reshape(-1, 3), np.broadcast_to(n, ((H - 1) * (W - 1), 3)), atol=2e-4)


def _scene(n_fused=5):
    seq = synth.sequence_tracking(n_frames=n_fused + 3)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=8)
    for f in range(n_fused):
        d, _ = seq.frame(f)
        o.integrate_geometry(d, seq.K_depth, seq.poses[f])
    return seq, o


@pytest.fixture(scope="module")
def scene():
    return _scene()


def pose_error(A, B):
    A, B = np.asarray(A, np.float64), np.asarray(B, np.float64)
    R = A[:3, :3].T @ B[:3, :3]
    return 1e3 * np.linalg.norm(A[:3, 3] - B[:3, 3]), math.degrees(math.acos(min(1.0, max(-1.0, (np.trace(R) - 1) / 2))))


@pytest.mark.parametrize("frame", [5, 6])
def test_tracking_recovers_the_true_pose(scene, frame):
    """Frame k tracked against the volume fused from frames 0..4, starting
    from the previous frame's true pose (2 deg of orbit plus 2 mm / 0.2 deg of
    jitter away): the result is within 1 mm and 0.1 deg of frame k's pose."""
    seq, o = scene
    d, _ = seq.frame(frame)
    T, log = oracle.track(o.F, o.W, seq.voxel_size, o.p.origin, seq.mu, d, seq.K_depth, seq.poses[frame - 1],
                          seq.poses[frame - 1])
    e0 = pose_error(seq.poses[frame - 1], seq.poses[frame])
    e1 = pose_error(T, seq.poses[frame])
    assert e0[0] > 10 and e0[1] > 1.0
    assert e1[0] < 1.0 and e1[1] < 0.1, (e0, e1)
    assert [r["level"] for r in log] == [2] * 4 + [1] * 5 + [0] * 10
    assert all(r["n"] > 5000 for r in log)
    # the residual falls from the first to the last iteration of the coarsest level
    assert log[3]["err2"] / log[3]["n"] < 0.25 * log[0]["err2"] / log[0]["n"]


def test_normal_equations_equal_a_binary64_evaluation(scene):
    """A and g of one level at a perturbed pose, against the same sums
    evaluated in binary64 numpy from the maps (pixels whose association or
    gates lie within rounding of a threshold are left out on both sides)."""
    seq, o = scene
    d, _ = seq.frame(5)
    l = 1
    Kl = oracle.icp_level_K(seq.K_depth, l)
    pyr = oracle.icp_pyramid(d, 3)
    h, w = pyr[l].shape
    Tp = seq.poses[4]
    pred = oracle.raycast(o.F, o.W, None, seq.voxel_size, seq.voxel_size, o.p.origin, Kl, Tp, (w, h), 0.1, 4.0,
                          mu=seq.mu)
    V, N = oracle.icp_maps(pyr[l], Kl)
    Tc = np.asarray(seq.poses[4], np.float64)
    r = oracle.icp_system(V, N, pred["vertex"], pred["normal"], Kl, Tc, Tp)
    # numpy, binary64 from the binary32 inputs
    Tc32 = Tc.astype(np.float32).astype(np.float64)
    R, t = Tc32[:3, :3], Tc32[:3, 3]
    Tp64 = np.asarray(Tp, np.float64)
    Rp, tp = Tp64[:3, :3].T, -(Tp64[:3, :3].T @ Tp64[:3, 3])
    Vf, Nf = V.reshape(-1, 3).astype(np.float64), N.reshape(-1, 3).astype(np.float64)
    ok = (Vf[:, 2] != 0) & np.any(Nf != 0, axis=1)
    p = Vf @ R.T + t
    m = Nf @ R.T
    qc = p @ Rp.T + tp
    with np.errstate(divide="ignore", invalid="ignore"):
        ux = Kl[0, 0] * qc[:, 0] / qc[:, 2] + Kl[0, 2]
        uy = Kl[1, 1] * qc[:, 1] / qc[:, 2] + Kl[1, 2]
    fu, fv = np.floor(ux + 0.5), np.floor(uy + 0.5)
    tie = (np.abs(ux + 0.5 - np.round(ux + 0.5)) < 1e-3) | (np.abs(uy + 0.5 - np.round(uy + 0.5)) < 1e-3)
    ok &= (qc[:, 2] > 0) & (fu >= 0) & (fu <= w - 1) & (fv >= 0) & (fv <= h - 1)
    j = np.where(ok, fv * w + fu, 0).astype(np.int64)
    q = pred["vertex"].reshape(-1, 3).astype(np.float64)[j]
    nq = pred["normal"].reshape(-1, 3).astype(np.float64)[j]
    ok &= np.any(nq != 0, axis=1)
    e = p - q
    dist2 = (e * e).sum(1)
    cosang = (m * nq).sum(1)
    tie |= (np.abs(dist2 - oracle.ICP_MAX_DIST ** 2) < 1e-6) | (np.abs(cosang - oracle.ICP_MIN_COS) < 1e-5)
    ok &= (dist2 <= oracle.ICP_MAX_DIST ** 2) & (cosang >= oracle.ICP_MIN_COS)
    res = (e * nq).sum(1)
    Jall = np.concatenate([nq, np.cross(p, nq)], 1)
    sure, maybe = ok & ~tie, tie & np.isfinite(res)
    assert maybe.sum() < 20  # a handful of pixels near a threshold, decided either way
    J = Jall[sure]
    A = J.T @ J
    g = J.T @ res[sure]
    Jm = np.nan_to_num(Jall[maybe])
    slack_A = np.abs(Jm).T @ np.abs(Jm)
    slack_g = np.abs(Jm).T @ np.abs(np.nan_to_num(res[maybe]))
    assert int(sure.sum()) <= r["n"] <= int(sure.sum() + maybe.sum()) and r["n"] > 10000
    assert np.all(np.abs(r["A"] - A) <= slack_A + 1e-5 * np.abs(A) + 1e-6 * np.abs(A).max())
    assert np.all(np.abs(r["g"] - g) <= slack_g + 1e-4 * np.abs(g) + 1e-5 * np.abs(g).max())


def test_a_single_plane_leaves_three_directions_unconstrained(oracle_lib):
    """Point-to-plane ICP against a plane constrains only the translation
    along its normal and the rotations about the two in-plane axes: A has
    rank 3, its null space spans the in-plane translations and the rotation
    about the normal (taken about the world origin)."""
    W, H = 80, 60
    K = K_of(70.0, W, H)
    d = np.full((H, W), 1.0, np.float32)
    V, N = oracle.icp_maps(d, K)
    T = np.eye(4)  # camera = world; the plane is z = 1, normal (0, 0, -1)
    r = oracle.icp_system(V, N, V, N, K, T, T)
    assert r["n"] > 4000 and r["err2"] == 0.0
    ev = np.linalg.eigvalsh(r["A"])
    assert ev[2] < 1e-9 * ev[-1] and ev[3] > 1e-4 * ev[-1]
    A = r["A"]
    for v in (np.array([1.0, 0, 0, 0, 0, 0]), np.array([0, 1.0, 0, 0, 0, 0]), np.array([0, 0, 0, 0, 0, 1.0])):
        assert np.linalg.norm(A @ v) < 1e-9 * np.linalg.norm(A)


def test_pose_update_is_the_left_exponential(oracle_lib):
    xi = np.array([0.01, -0.02, 0.005, 0.03, -0.01, 0.02])
    T0 = np.eye(4)
    T0[:3, 3] = [0.1, 0.2, -0.3]
    T1 = oracle.icp_update(xi, T0)
    from paper_1602_06645_gb300.adjoint import se3_exp
    np.testing.assert_allclose(T1, se3_exp(xi) @ T0, atol=1e-12)
