"""GPU adjoint (photometric colour loss) against the binary64 oracle.

The recorded gate sets S_k must equal the oracle's exactly (they come from
the same binary32 gates); the binary32 forward colours and the gradients with
respect to K_hd, the se(3) extrinsic and the HD pixels must match the oracle's
binary64 values within a relative error of 1e-3 (for the ten camera
parameters: of the gradient vector, and per component against
max(|g_j|, 0.1 max|g|), since small components are sums with cancellation).
The bilinear cell of each sample is an integer decision, so the oracle takes it
in binary32 with the kernels' operation order.
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
from paper_1602_06645_gb300.adjoint import Adjoint, fuse_colours, se3_exp  # noqa: E402

REL = 1e-3


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


@pytest.fixture(scope="module", params=[(32, 4, 160, 120), (48, 6, 320, 240)])
def setup(request):
    dims_geo, n_frames, cw, ch = request.param
    seq = synth.sequence_adjoint(n_frames=n_frames, seed=4, dims_geo=dims_geo)
    seq.rgb_size = (cw, ch)
    seq.K_rgb = synth.intrinsics(1050.0 * cw / 1920, 1050.0 * cw / 1920, (cw - 1) / 2.0, (ch - 1) / 2.0)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    adj = Adjoint(vol, max_frames=n_frames, max_pairs=1 << 22)
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
    T0 = perturbed(seq.T_depth_rgb)
    th0 = np.concatenate([Ktrue * np.array([1.01, 0.99, 1.0, 1.0]) + np.array([0, 0, 0.7, -0.4]), np.zeros(6)])
    truth = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), seq.T_depth_rgb)
    th_true = np.concatenate([Ktrue, np.zeros(6)])
    tg = truth.eval(th_true, truth.cells(th_true))
    target = np.where(tg["n"][:, None] > 0, tg["C"], np.nan)
    orc = oracle.Adjoint(imgs, Rn, tn, S, seq.dims_col, o.p.s_c, list(o.p.origin), T0)
    yield dict(seq=seq, S=S, adj=adj, vol=vol, nv=nv, imgs=imgs, T0=T0, th0=th0, orc=orc, target=target)
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


def test_forward_colours_match_binary64(setup):
    st = setup
    th0 = st["th0"]
    T = (se3_exp(th0[4:]) @ st["T0"]).astype(np.float32)
    C, n = st["adj"].forward(torch.from_numpy(st["imgs"]).cuda(), th0[:4].astype(np.float32), T)
    pos = gpu_order(st)
    ref = st["orc"].eval(th0, st["orc"].cells32(th0[:4], T))
    Cg = np.empty_like(ref["C"])
    ng = np.empty_like(ref["n"])
    Cg[pos] = C.cpu().numpy()
    ng[pos] = n.cpu().numpy()
    same = ng == ref["n"]
    assert same.mean() > 0.999
    err = np.abs(Cg[same] - ref["C"][same])
    assert np.quantile(err, 0.999) < 0.05 and err.mean() < 1e-3


def test_backward_gradients_match_binary64(setup):
    st = setup
    th0, orc = st["th0"], st["orc"]
    T = (se3_exp(th0[4:]) @ st["T0"]).astype(np.float32)
    k4 = th0[:4].astype(np.float32)
    images = torch.from_numpy(st["imgs"]).cuda()
    C, n = st["adj"].forward(images, k4, T)
    pos = gpu_order(st)
    tgt = np.nan_to_num(st["target"][pos].astype(np.float32), nan=0.0)
    has_t = torch.from_numpy(~np.isnan(st["target"][pos][:, 0])).cuda()
    grad_C = 2.0 * (C - torch.from_numpy(tgt).cuda()) * has_t[:, None]
    gI = torch.zeros_like(images)
    g = st["adj"].backward(images, k4, T, grad_C.contiguous(), gI)
    cells = orc.cells32(k4, T)  # the cell choice is an integer decision: binary32 on both sides
    ref = orc.eval(th0, cells, st["target"], grad=True)
    # relative error of the gradient vector; per component against max(|g_j|, 0.1 |g|_inf)
    assert np.linalg.norm(g - ref["grad"]) <= REL * np.linalg.norm(ref["grad"])
    scale = np.abs(ref["grad"])
    for j in range(10):
        assert abs(g[j] - ref["grad"][j]) <= REL * max(scale[j], 0.1 * scale.max()), (j, g[j], ref["grad"][j])
    # pixel gradients: sample pixel channels with a non-negligible gradient
    gIc = gI.cpu().numpy()
    idx = np.argwhere(np.abs(gIc) > 1e-3 * np.abs(gIc).max())
    rng = np.random.default_rng(3)
    pick = idx[rng.choice(len(idx), size=min(48, len(idx)), replace=False)]
    q = orc.eval(th0, cells, st["target"], query=pick)["qgrad"]
    got = gIc[tuple(pick.T)]
    rel = np.abs(got - q) / np.maximum(np.abs(q), 1e-3 * np.abs(gIc).max())
    assert np.quantile(rel, 0.95) <= REL and rel.max() < 0.05


def test_autograd_function(setup):
    st = setup
    images = torch.from_numpy(st["imgs"]).cuda().requires_grad_(True)
    K4 = torch.tensor(st["th0"][:4], dtype=torch.float64, requires_grad=True)
    xi = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    C, n = fuse_colours(images, K4, xi, st["adj"], st["T0"])
    pos = gpu_order(st)
    tgt = torch.from_numpy(np.nan_to_num(st["target"][pos], nan=0.0).astype(np.float32)).cuda()
    mask = torch.from_numpy(~np.isnan(st["target"][pos][:, 0])).cuda() & (n > 0)
    loss = (((C - tgt) ** 2).sum(dim=1) * mask).sum()
    loss.backward()
    T = (se3_exp(np.zeros(6)) @ st["T0"]).astype(np.float32)
    ref = st["orc"].eval(st["th0"], st["orc"].cells32(st["th0"][:4], T), st["target"], grad=True)
    assert abs(loss.item() - ref["loss"]) <= 1e-3 * ref["loss"]
    g = np.concatenate([K4.grad.numpy(), xi.grad.numpy()])
    assert np.linalg.norm(g - ref["grad"]) <= REL * np.linalg.norm(ref["grad"])
    assert images.grad is not None and float(images.grad.abs().sum()) > 0
