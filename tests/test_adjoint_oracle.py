"""Pins of the binary64 adjoint oracle (photometric colour loss and its
gradient with respect to the HD intrinsics, the se(3) extrinsic and the HD
pixels).

The analytic gradient must agree with central finite differences of the loss
(binary64, step 1e-6, the discrete choices held fixed); the depth-side gate
sets must be exactly the voxels the fusion step can colour.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1602_06645_gb300 import synth


def small_problem(n_frames=4, dims_geo=32, cw=160, ch=120, seed=4):
    seq = synth.sequence_adjoint(n_frames=n_frames, seed=seed, dims_geo=dims_geo)
    seq.rgb_size = (cw, ch)
    seq.K_rgb = synth.intrinsics(1050.0 * cw / 1920, 1050.0 * cw / 1920, (cw - 1) / 2.0, (ch - 1) / 2.0)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    S, imgs, Rn, tn = [], [], [], []
    for f in range(n_frames):
        d, c = seq.frame(f)
        S.append(o.record_gates(d, seq.K_depth, seq.poses[f]))
        imgs.append(c.astype(np.float32))
        R, t, _ = o.frame_constants(seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        Rn.append(R)
        tn.append(t)
    return seq, o, S, np.stack(imgs), np.stack(Rn), np.stack(tn)


def perturbed(T, seed=0, dt=0.01, deg=1.0):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    b = rng.normal(size=3)
    b /= np.linalg.norm(b)
    P = np.eye(4)
    P[:3, :3] = synth.rot_axis_angle(b, math.radians(deg))
    P[:3, 3] = dt * a
    return P @ np.asarray(T, np.float64)


@pytest.fixture(scope="module")
def prob():
    seq, o, S, imgs, Rn, tn = small_problem()
    Ktrue = np.array([seq.K_rgb[0, 0], seq.K_rgb[1, 1], seq.K_rgb[0, 2], seq.K_rgb[1, 2]], np.float64)
    truth = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), seq.T_depth_rgb)
    th_true = np.concatenate([Ktrue, np.zeros(6)])
    tgt = truth.eval(th_true, truth.cells(th_true))
    target = np.where(tgt["n"][:, None] > 0, tgt["C"], np.nan)
    adj = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), perturbed(seq.T_depth_rgb))
    th0 = np.concatenate([Ktrue * np.array([1.01, 0.99, 1.0, 1.0]) + np.array([0, 0, 0.7, -0.4]), np.zeros(6)])
    return dict(seq=seq, o=o, S=S, adj=adj, truth=truth, th0=th0, th_true=th_true, target=target)


def test_gate_sets_are_non_trivial(prob):
    assert all(len(s) > 200 for s in prob["S"])
    assert len(prob["adj"].V) > 500


def test_theta_gradient_matches_central_differences(prob):
    adj, th0, target = prob["adj"], prob["th0"], prob["target"]
    cells = adj.cells(th0)
    r = adj.eval(th0, cells, target, grad=True)
    assert r["loss"] > 0
    g = r["grad"]
    for j in range(10):
        h = 1e-6 * max(1.0, abs(th0[j]))
        tp, tm = th0.copy(), th0.copy()
        tp[j] += h
        tm[j] -= h
        fd = (adj.eval(tp, cells, target)["loss"] - adj.eval(tm, cells, target)["loss"]) / (2 * h)
        scale = max(abs(g[j]), 1e-6 * np.abs(g).max())
        assert abs(fd - g[j]) <= 1e-5 * scale, (j, fd, g[j])


def test_pixel_gradient_matches_central_differences(prob):
    adj, th0, target = prob["adj"], prob["th0"], prob["target"]
    cells = adj.cells(th0)
    valid = cells[0::2] != np.iinfo(np.int32).min
    rng = np.random.default_rng(7)
    # pixels under samples of frames 0..3: pick 24 pairs, one corner channel each
    offs = adj.offsets
    pairs = rng.choice(np.nonzero(valid)[0], size=24, replace=False)
    query = []
    for i in pairs:
        k = int(np.searchsorted(offs, i, side="right") - 1)
        x0, y0 = cells[2 * i], cells[2 * i + 1]
        query.append((k, y0 + int(rng.integers(0, 2)), x0 + int(rng.integers(0, 2)), int(rng.integers(0, 3))))
    query = np.array(query, np.int64)
    qg = adj.eval(th0, cells, target, query=query)["qgrad"]
    h = 1e-2
    for q, g in zip(query, qg):
        k, y, x, c = q
        base = adj.images[k, y, x, c]
        up, dn = np.float32(base + h), np.float32(base - h)  # the binary32 values actually applied
        adj.images[k, y, x, c] = up
        lp = adj.eval(th0, cells, target)["loss"]
        adj.images[k, y, x, c] = dn
        lm = adj.eval(th0, cells, target)["loss"]
        adj.images[k, y, x, c] = base
        fd = (lp - lm) / (float(up) - float(dn))
        # L is quadratic in each intensity: the central difference is exact up to rounding
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (q, fd, g)


def test_truth_has_zero_loss_and_gradient(prob):
    tr, th, target = prob["truth"], prob["th_true"], prob["target"]
    r = tr.eval(th, tr.cells(th), target, grad=True)
    assert r["loss"] == 0.0
    assert np.all(r["grad"] == 0.0)


def test_gradient_step_on_the_extrinsic_reduces_the_loss(prob):
    adj, th0, target = prob["adj"], prob["th0"], prob["target"]
    th = th0.copy()
    th[:4] = prob["th_true"][:4]
    cells = adj.cells(th)
    r = adj.eval(th, cells, target, grad=True)
    step = np.zeros(10)
    step[4:] = -r["grad"][4:] / np.linalg.norm(r["grad"][4:])
    best = min(adj.eval(th + a * step, cells, target)["loss"] for a in (1e-5, 1e-4, 1e-3))
    assert best < r["loss"]


def test_gate_sets_are_the_colourable_voxels(prob):
    """S_k holds every voxel the fusion step colours in frame k (with an HD
    image large enough to see them all) and nothing else."""
    seq = prob["seq"]
    big = (640, 480)
    K = synth.intrinsics(300.0, 300.0, 319.5, 239.5)
    o1 = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, 255)
    o2 = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, 255)
    rgb = np.full((big[1], big[0], 3), 100, np.uint8)
    prev = np.zeros_like(o1.C)
    for f in range(len(prob["S"])):
        d, _ = seq.frame(f)
        o1.integrate(d, rgb, seq.K_depth, K, seq.poses[f], seq.T_depth_rgb)
        S = o2.record_gates(d, seq.K_depth, seq.poses[f])
        updated = np.nonzero((o1.C != prev).ravel())[0]
        prev = o1.C.copy()
        assert np.array_equal(np.sort(updated), S) or set(updated.tolist()) <= set(S.tolist())
        missing = set(S.tolist()) - set(updated.tolist())
        assert len(missing) <= max(2, len(S) // 100)  # only voxels whose HD footprint leaves the image


def test_forward_of_linear_images_is_the_mean_projected_pixel(prob):
    """Bilinear interpolation reproduces a linear image exactly, so with HD
    images I_k(x, y) = a_k x + b_k y + c_k the fused colour of a voxel is the
    mean over its in-image frames of a_k u_k + b_k v_k + c_k, where (u_k, v_k)
    is the voxel centre moved by (R_n, t_n) (Eq. 5), by the extrinsic T0
    (Eq. 3) and projected with K_hd (Eq. 4) — computed here in numpy."""
    seq, o, S, adj = prob["seq"], prob["o"], prob["S"], prob["adj"]
    n, H, W, _ = adj.images.shape
    ab = np.array([[0.5, 0.25, 3.0], [-0.125, 0.75, 90.0], [0.3125, -0.0625, 40.0]])  # per channel
    xs, ys = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    imgs = np.stack([np.stack([ab[c, 0] * xs + ab[c, 1] * ys + ab[c, 2] + 7.0 * k for c in range(3)], -1)
                     for k in range(n)]).astype(np.float32)
    lin = oracle.Adjoint(imgs, adj.Rn, adj.tn, S, seq.dims_col, o.p.s_c, list(o.p.origin),
                         np.asarray(perturbed(seq.T_depth_rgb)))
    th = prob["th0"]
    r = lin.eval(th, lin.cells(th))
    # numpy: voxel centres -> depth camera -> HD camera -> pixel
    nc = seq.dims_col
    V = lin.V.astype(np.int64)
    ijk = np.stack([V % nc[0], (V // nc[0]) % nc[1], V // (nc[0] * nc[1])], 1).astype(np.float64)
    pw = np.asarray(o.p.origin, np.float64) + (ijk + 0.5) * np.float64(o.p.s_c)
    T0 = np.asarray(perturbed(seq.T_depth_rgb), np.float64)
    fx, fy, cx, cy = th[:4]
    acc = np.zeros((len(V), 3))
    cnt = np.zeros(len(V), np.int64)
    for k in range(n):
        members = np.isin(lin.V, S[k])
        Pc = pw @ adj.Rn[k].reshape(3, 3).astype(np.float64).T + adj.tn[k].astype(np.float64)
        Ph = Pc @ T0[:3, :3].T + T0[:3, 3]
        u, v = fx * Ph[:, 0] / Ph[:, 2] + cx, fy * Ph[:, 1] / Ph[:, 2] + cy
        inside = members & (np.floor(u) >= 0) & (np.floor(u) + 1 <= W - 1) & (np.floor(v) >= 0) & \
            (np.floor(v) + 1 <= H - 1)
        val = ab[:, 0][None, :] * u[:, None] + ab[:, 1][None, :] * v[:, None] + ab[:, 2][None, :] + 7.0 * k
        acc[inside] += val[inside]
        cnt += inside
    ok = cnt > 0
    assert ok.sum() > 1000
    # the count of in-image frames may differ only for samples within rounding of the image border
    assert (r["n"][ok] == cnt[ok]).mean() > 0.999
    same = ok & (r["n"] == cnt)
    np.testing.assert_allclose(r["C"][same], acc[same] / cnt[same, None], rtol=0, atol=1e-4)


# ------------------------------------------------ bilinear cells (binary32) --
def _cells64(adj, K4, T, W, H):
    """Binary64 cells of every pair: the voxel centre moved by (R_n, t_n)
    (Eq. 5) and by T (Eq. 3), projected with (fx, fy, cx, cy) (Eq. 4); the
    footprint (x0..x0+1, y0..y0+1) must lie in the W x H image.  Also returns
    the distance of u and v from the nearest integer (the near-tie margin)."""
    nc = np.array(adj.p.nc, np.int64)
    org = np.array(adj.p.origin, np.float64)
    s = float(np.float32(adj.p.s_c))
    fx, fy, cx, cy = [float(v) for v in np.asarray(K4, np.float32)]
    T = np.asarray(T, np.float32).astype(np.float64)
    x0 = np.full(len(adj.idx), np.iinfo(np.int32).min, np.int64)
    y0 = x0.copy()
    margin = np.full(len(adj.idx), np.inf)
    for k in range(len(adj.offsets) - 1):
        sl = slice(adj.offsets[k], adj.offsets[k + 1])
        v = adj.idx[sl].astype(np.int64)
        ijk = np.stack([v % nc[0], (v // nc[0]) % nc[1], v // (nc[0] * nc[1])], 1).astype(np.float64)
        pw = org + (ijk + 0.5) * s
        Pc = pw @ adj.Rn[k].reshape(3, 3).astype(np.float64).T + adj.tn[k].astype(np.float64)
        Ph = Pc @ T[:3, :3].T + T[:3, 3]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * Ph[:, 0] / Ph[:, 2] + cx
            w = fy * Ph[:, 1] / Ph[:, 2] + cy
        fu, fw = np.floor(u), np.floor(w)
        ok = (Ph[:, 2] > 0) & (fu >= 0) & (fu <= W - 2) & (fw >= 0) & (fw <= H - 2)
        x0[sl] = np.where(ok, fu, x0[sl])
        y0[sl] = np.where(ok, fw, y0[sl])
        margin[sl] = np.minimum(np.abs(u - np.round(u)), np.abs(w - np.round(w)))
    return x0, y0, margin


def test_cells_equal_binary64_cells_away_from_ties(prob):
    """The binary32 cell decision (the fusion oracle's colour path) equals the
    binary64 floor of the projected sample wherever u and v are farther than
    1e-3 pixel from an integer."""
    adj, th0, seq = prob["adj"], prob["th0"], prob["seq"]
    _, H, W, _ = adj.images.shape
    K4 = (th0[:4] - np.array([0.0, 0.0, 0.3 * W, 0.0])).astype(np.float32)  # part of the scan leaves the image
    T = np.asarray(perturbed(seq.T_depth_rgb), np.float32)
    cells = adj.cells32(K4, T)
    x0, y0, margin = _cells64(adj, K4, T, W, H)
    far = margin > 1e-3
    assert far.mean() > 0.99
    np.testing.assert_array_equal(cells[0::2][far], x0[far])
    np.testing.assert_array_equal(cells[1::2][far], y0[far])
    valid = cells[0::2] != np.iinfo(np.int32).min
    assert valid.sum() > 1000 and (~valid).sum() > 10  # the case has samples on both sides of the border


def test_cells_equal_binary64_cells_full_hd(prob):
    """The same at the HD camera of the rig (1920 x 1080, f = 1050): most
    samples now fall inside the image."""
    seq, o, S = prob["seq"], prob["o"], prob["S"]
    adj = prob["adj"]
    n = len(S)
    imgs = np.zeros((n, 1080, 1920, 3), np.float32)
    big = oracle.Adjoint(imgs, adj.Rn, adj.tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), np.eye(4))
    K4 = np.array([1050.0, 1050.0, 959.5, 539.5], np.float32)
    T = np.asarray(perturbed(seq.T_depth_rgb, seed=5), np.float32)
    cells = big.cells32(K4, T)
    x0, y0, margin = _cells64(big, K4, T, 1920, 1080)
    far = margin > 1e-3
    np.testing.assert_array_equal(cells[0::2][far], x0[far])
    np.testing.assert_array_equal(cells[1::2][far], y0[far])
    assert (cells[0::2] != np.iinfo(np.int32).min).mean() > 0.5


def test_cells_at_the_image_edge():
    """Samples placed exactly (dyadic values) on either side of the image
    border: the 2x2 footprint (x0..x0+1, y0..y0+1) must lie inside the
    16 x 12 image, x0 = floor(u) (not the nearest integer), u = fx X / Z + cx."""
    Wd, Hd = 16, 12
    fx, fy, cx, cy = 2.0, 2.0, 3.0, 1.0
    # one colour voxel (centre (0.125, 0.125, 0.125)) seen in one frame per case
    us = [(-0.25, 5.0), (0.0, 5.0), (0.75, 5.0), (14.0, 5.0), (15.0 - 2.0 ** -10, 5.0), (15.0, 5.0),
          (5.0, -0.5), (5.0, 0.0), (5.0, 10.0), (5.0, 10.5), (5.0, 11.0), (3.25, 7.5)]
    want = [None, (0, 5), (0, 5), (14, 5), (14, 5), None, None, (5, 0), (5, 10), (5, 10), None, (3, 7)]
    n = len(us)
    Rn = np.tile(np.eye(3, dtype=np.float32).reshape(9), (n, 1))
    tn = np.array([[(u - cx) / fx - 0.125, (v - cy) / fy - 0.125, 1.0 - 0.125] for u, v in us], np.float32)
    S = [np.zeros(1, np.uint32) for _ in range(n)]
    imgs = np.zeros((n, Hd, Wd, 3), np.float32)
    adj = oracle.Adjoint(imgs, Rn, tn, S, (1, 1, 1), 0.25, [0.0, 0.0, 0.0], np.eye(4))
    cells = adj.cells32(np.array([fx, fy, cx, cy], np.float32), np.eye(4, dtype=np.float32))
    none = np.iinfo(np.int32).min
    got = [None if cells[2 * i] == none else (int(cells[2 * i]), int(cells[2 * i + 1])) for i in range(n)]
    assert got == want
