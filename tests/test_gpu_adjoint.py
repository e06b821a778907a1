"""GPU adjoint (photometric colour loss) against the binary64 oracle.

Both sides evaluate the same camera: the binary32 K_hd and T_depth_rgb the
kernels are given, read exactly as binary64 by the oracle (xi = 0).  Checks:

* the recorded gate sets S_k equal the oracle's exactly (the same binary32
  gates);
* the sample counts n_v equal the oracle's exactly (the bilinear footprint
  test is an integer decision, taken by the oracle on its fusion path);
* every forward colour is within 1e-3 of the binary64 mean, relative to
  max(|C|, 1);
* fed the same dL/dC (the binary32 value of the oracle's 2 (C - target)), the
  ten camera gradients are within 1e-3 of the oracle's (per component against
  max(|g_j|, 0.1 max|g|), since small components are sums with cancellation)
  and sampled pixel gradients within 1e-3 (against max(|g|, 1e-3 max|gI|)).

Cases: two small ones and the workload the benchmark times (256^3 geometry /
512^3 colour, 20 frames of 640x480 depth and 1920x1080 RGB, bilinear).
"""
import math
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1602_06645_gb300 as T  # noqa: E402
from paper_1602_06645_gb300 import synth  # noqa: E402
from paper_1602_06645_gb300.adjoint import Adjoint, fuse_colours  # noqa: E402

REL = 1e-3
CASES = {
    "32_160x120": (32, 4, (160, 120)),
    "48_320x240": (48, 6, (320, 240)),
    "256_512_1920x1080": (256, 20, None),  # the adjoint workload itself
}


def perturbed(Tm, seed=0, dt=0.01, deg=1.0):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    b = rng.normal(size=3)
    b /= np.linalg.norm(b)
    P = np.eye(4)
    P[:3, :3] = synth.rot_axis_angle(b, math.radians(deg))
    P[:3, 3] = dt * a
    return P @ np.asarray(Tm, np.float64)


@pytest.fixture(scope="module", params=sorted(CASES))
def setup(request):
    dims_geo, n_frames, rgb = CASES[request.param]
    seq = synth.sequence_adjoint(n_frames=n_frames, seed=4, dims_geo=dims_geo)
    if rgb is not None:
        cw, ch = rgb
        seq.rgb_size = (cw, ch)
        seq.K_rgb = synth.intrinsics(1050.0 * cw / 1920, 1050.0 * cw / 1920, (cw - 1) / 2.0, (ch - 1) / 2.0)
    nt = os.cpu_count() or 1
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=nt)
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    adj = Adjoint(vol, max_frames=n_frames, max_pairs=1 << 26)
    S, imgs, Rn, tn = [], [], [], []
    for f in range(n_frames):
        d, c = seq.frame(f)
        S.append(o.record_gates(d, seq.K_depth, seq.poses[f]))
        adj.record(torch.from_numpy(d.view(np.int16)).cuda(), seq.K_depth, seq.poses[f])
        imgs.append(c.astype(np.float32))
        R, t, _ = o.frame_constants(seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        Rn.append(R)
        tn.append(t)
    nv = adj.finalize()
    imgs = np.stack(imgs)
    Ktrue = np.array([seq.K_rgb[0, 0], seq.K_rgb[1, 1], seq.K_rgb[0, 2], seq.K_rgb[1, 2]], np.float64)
    # the camera both sides evaluate: binary32 values, read exactly in binary64
    k4 = (Ktrue * np.array([1.01, 0.99, 1.0, 1.0]) + np.array([0, 0, 0.7, -0.4])).astype(np.float32)
    T32 = perturbed(seq.T_depth_rgb).astype(np.float32)
    th = np.concatenate([k4.astype(np.float64), np.zeros(6)])
    truth = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), seq.T_depth_rgb)
    th_true = np.concatenate([Ktrue, np.zeros(6)])
    tg = truth.eval(th_true, truth.cells(th_true))
    target = np.where(tg["n"][:, None] > 0, tg["C"], np.nan)
    orc = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), T32.astype(np.float64))
    cells = orc.cells32(k4, T32)
    ref = orc.eval(th, cells)
    images = torch.from_numpy(imgs).cuda()
    yield dict(seq=seq, S=S, adj=adj, vol=vol, nv=nv, imgs=imgs, images=images, k4=k4, T32=T32, th=th, orc=orc,
               cells=cells, ref=ref, target=target)
    adj.close()
    vol.close()


def gpu_order(st):
    """Map from GPU slots to the oracle's (ascending) voxel order."""
    V = st["adj"].voxels.cpu().numpy().view(np.uint32)
    pos = np.searchsorted(st["orc"].V, V)
    assert np.array_equal(st["orc"].V[pos], V)
    return pos


def test_recorded_gate_sets_equal_the_oracle(setup):
    vox, fr = setup["adj"].pairs()
    for k, Sk in enumerate(setup["S"]):
        np.testing.assert_array_equal(np.sort(vox[fr == k]), Sk)
    assert setup["nv"] == len(setup["orc"].V)
    assert setup["nv"] > 1000


def test_forward_counts_and_colours_match_binary64(setup):
    st = setup
    C, n = st["adj"].forward(st["images"], st["k4"], st["T32"])
    pos = gpu_order(st)
    ref = st["ref"]
    Cg = np.empty_like(ref["C"])
    ng = np.empty_like(ref["n"])
    Cg[pos] = C.cpu().numpy()
    ng[pos] = n.cpu().numpy()
    np.testing.assert_array_equal(ng, ref["n"])
    assert (ref["n"] > 0).mean() > 0.5
    rel = np.abs(Cg - ref["C"]) / np.maximum(np.abs(ref["C"]), 1.0)
    assert rel.max() <= REL, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))


def _same_grad_C(st, pos):
    """dL/dC given to both sides: the binary32 value of the oracle's
    2 (C - target) on voxels with a target, 0 elsewhere; and the target that
    makes the oracle's own 2 (C - target) equal to it."""
    ref = st["ref"]
    has_t = ~np.isnan(st["target"][:, 0]) & (ref["n"] > 0)
    g = np.where(has_t[:, None], 2.0 * (ref["C"] - np.nan_to_num(st["target"])), 0.0).astype(np.float32)
    tgt = np.where(has_t[:, None], ref["C"] - 0.5 * g.astype(np.float64), np.nan)
    return torch.from_numpy(np.ascontiguousarray(g[pos])).cuda(), tgt


def test_backward_gradients_match_binary64(setup):
    st = setup
    orc = st["orc"]
    st["adj"].forward(st["images"], st["k4"], st["T32"])
    pos = gpu_order(st)
    gC, tgt = _same_grad_C(st, pos)
    gI = torch.zeros_like(st["images"])
    g = st["adj"].backward(st["images"], st["k4"], st["T32"], gC, gI)
    ref = orc.eval(st["th"], st["cells"], tgt, grad=True)
    assert np.linalg.norm(g - ref["grad"]) <= REL * np.linalg.norm(ref["grad"])
    scale = np.abs(ref["grad"])
    for j in range(10):
        assert abs(g[j] - ref["grad"][j]) <= REL * max(scale[j], 0.1 * scale.max()), (j, g[j], ref["grad"][j])
    # pixel gradients: sampled pixel channels with a non-negligible gradient
    gIc = gI.cpu().numpy()
    idx = np.argwhere(np.abs(gIc) > 1e-3 * np.abs(gIc).max())
    rng = np.random.default_rng(3)
    pick = idx[rng.choice(len(idx), size=min(64, len(idx)), replace=False)]
    q = orc.eval(st["th"], st["cells"], tgt, query=pick)["qgrad"]
    got = gIc[tuple(pick.T)]
    rel = np.abs(got - q) / np.maximum(np.abs(q), 1e-3 * np.abs(gIc).max())
    assert rel.max() <= REL, (rel.max(), pick[rel.argmax()])


def test_autograd_function(setup):
    st = setup
    images = st["images"].clone().requires_grad_(True)
    K4 = torch.tensor(st["k4"].astype(np.float64), dtype=torch.float64, requires_grad=True)
    xi = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    C, n = fuse_colours(images, K4, xi, st["adj"], st["T32"])
    pos = gpu_order(st)
    tgt = torch.from_numpy(np.nan_to_num(st["target"][pos], nan=0.0).astype(np.float32)).cuda()
    mask = torch.from_numpy(~np.isnan(st["target"][pos][:, 0])).cuda() & (n > 0)
    loss = (((C - tgt) ** 2).sum(dim=1) * mask).sum()
    loss.backward()
    ref = st["orc"].eval(st["th"], st["cells"], st["target"], grad=True)
    assert abs(loss.item() - ref["loss"]) <= REL * ref["loss"]
    g = np.concatenate([K4.grad.numpy(), xi.grad.numpy()])
    assert np.linalg.norm(g - ref["grad"]) <= REL * np.linalg.norm(ref["grad"])
    assert images.grad is not None and float(images.grad.abs().sum()) > 0


def test_autograd_function_rejects_nonzero_xi(setup):
    st = setup
    xi = torch.full((6,), 1e-3, dtype=torch.float64, requires_grad=True)
    K4 = torch.tensor(st["k4"].astype(np.float64), dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError):
        fuse_colours(st["images"], K4, xi, st["adj"], st["T32"])
