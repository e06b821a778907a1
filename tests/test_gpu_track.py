"""GPU camera tracking (tsdf_track) against the oracle (oracle/icp.c).

Both sides track the same depth frame against the same geometry volume (the
oracle's fusion of the earlier frames, written into the GPU volume), from the
same starting pose.  For every step the GPU reports the pose it started from;
the oracle, given that pose, must find exactly the same correspondences and
the same normal equations (A, g within 1e-9 relative: only the binary64
summation order differs).  The final poses agree to 1e-6, and both recover
the frame's true pose (the sequence's ground truth) to 1 mm / 0.1 degree.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1602_06645_gb300 as T  # noqa: E402
from paper_1602_06645_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def scene():
    seq = synth.sequence_tracking(n_frames=9)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=8)
    for f in range(5):
        d, _ = seq.frame(f)
        o.integrate_geometry(d, seq.K_depth, seq.poses[f])
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    vol.write(o.F, o.W)
    yield seq, o, vol
    vol.close()


def pose_error(A, B):
    A, B = np.asarray(A, np.float64), np.asarray(B, np.float64)
    R = A[:3, :3].T @ B[:3, :3]
    return 1e3 * np.linalg.norm(A[:3, 3] - B[:3, 3]), math.degrees(math.acos(min(1.0, max(-1.0, (np.trace(R) - 1) / 2))))


@pytest.mark.parametrize("frame,host_depth", [(5, False), (6, True), (7, False)])
def test_tracking_steps_equal_the_oracle(scene, frame, host_depth):
    seq, o, vol = scene
    p = T.tsdf_track_params_default()
    d, _ = seq.frame(frame)
    depth = d if host_depth else torch.from_numpy(d.view(np.int16)).cuda()
    Tp = seq.poses[frame - 1]
    Tg, rep = T.tsdf_track(vol.h, depth, seq.K_depth, Tp, np.asarray(Tp, np.float64), p)
    iters = (p.iterations[0], p.iterations[1], p.iterations[2])
    To, log = oracle.track(o.F, o.W, seq.voxel_size, o.p.origin, seq.mu, d, seq.K_depth, Tp, Tp, levels=p.levels,
                           iterations=iters, max_dist=p.max_distance, min_cos=p.min_normal_cos, near=p.near_m,
                           far=p.far_m)
    assert rep.steps == len(log) == sum(iters)
    # every GPU step against the oracle's system at the GPU's pose
    pyr = oracle.icp_pyramid(d, p.levels)
    cache = {}
    for k in range(rep.steps):
        l = rep.level[k]
        assert l == log[k]["level"]
        if l not in cache:
            Kl = oracle.icp_level_K(seq.K_depth, l)
            h, w = pyr[l].shape
            pred = oracle.raycast(o.F, o.W, None, seq.voxel_size, seq.voxel_size, o.p.origin, Kl, Tp, (w, h),
                                  p.near_m, p.far_m, mu=seq.mu)
            cache[l] = (Kl, oracle.icp_maps(pyr[l], Kl), pred)
        Kl, (V, N), pred = cache[l]
        Tb = np.array(rep.T_before[k][:], np.float64).reshape(4, 4)
        r = oracle.icp_system(V, N, pred["vertex"], pred["normal"], Kl, Tb, Tp, p.max_distance, p.min_normal_cos)
        assert rep.correspondences[k] == r["n"] > 3000
        A = np.array(rep.A[k][:]).reshape(6, 6)
        g = np.array(rep.g[k][:])
        # sums of ~10^4 terms in another order: relative to each entry, or to the
        # largest entry where an entry is a sum with cancellation
        np.testing.assert_allclose(A, r["A"], rtol=1e-9, atol=1e-9 * np.abs(r["A"]).max())
        np.testing.assert_allclose(g, r["g"], rtol=1e-9, atol=1e-9 * np.abs(r["g"]).max())
        assert abs(rep.err2[k] - r["err2"]) <= 1e-9 * r["err2"]
        assert rep.solved[k] == 1
    np.testing.assert_allclose(Tg, To, atol=1e-6)
    e0, e1 = pose_error(Tp, seq.poses[frame]), pose_error(Tg, seq.poses[frame])
    assert e0[0] > 5 and e1[0] < 1.0 and e1[1] < 0.1, (e0, e1)


def test_tracking_arguments_are_checked(scene):
    seq, o, vol = scene
    d, _ = seq.frame(5)
    p = T.tsdf_track_params_default()
    p.levels = 4
    with pytest.raises(T.TsdfError):
        T.tsdf_track(vol.h, d, seq.K_depth, seq.poses[4], np.eye(4), p)
    p = T.tsdf_track_params_default()
    p.iterations[0] = 40
    with pytest.raises(T.TsdfError):
        T.tsdf_track(vol.h, d, seq.K_depth, seq.poses[4], np.eye(4), p)
    K = np.array(seq.K_depth, np.float32)
    K[0, 1] = 0.5  # skew: not a pinhole K
    with pytest.raises(T.TsdfError):
        T.tsdf_track(vol.h, d, K, seq.poses[4], np.eye(4))
