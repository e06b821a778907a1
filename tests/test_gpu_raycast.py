"""GPU ray caster (tsdf_raycast) against the ray-casting oracle.

The volumes the GPU casts come from outside the CUDA path: analytic signed
distances, or the oracle's own fusion of a synthetic sequence, written into
the GPU volume with tsdf_write.  Hit masks and colours must match bit for
bit; ranges, vertices and normals follow the same binary32 operations and
must match within 1e-5 (they are expected to be identical).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1602_06645_gb300 as T  # noqa: E402
from paper_1602_06645_gb300 import synth  # noqa: E402

TOL = 1e-5


def assert_same(gpu, orc, label=""):
    np.testing.assert_array_equal(gpu["range"] > 0, orc["range"] > 0, err_msg="hit mask " + label)
    np.testing.assert_array_equal(gpu["rgbw"].view(np.uint32), orc["rgbw"], err_msg="colour " + label)
    for k in ("range", "vertex", "normal"):
        d = np.abs(gpu[k] - orc[k])
        assert d.max() <= TOL, "%s differs by %g %s" % (k, d.max(), label)
    return float(np.mean([np.array_equal(gpu[k], orc[k]) for k in ("range", "vertex", "normal")]))


def analytic(kind, n=64):
    s = 1.0 / n
    c = -0.5 + (np.arange(n, dtype=np.float64) + 0.5) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    if kind == "plane":
        sd = z + 0.1
    else:
        sd = np.sqrt((x - 0.02) ** 2 + (y + 0.03) ** 2 + (z + 0.05) ** 2) - 0.22
    F = np.clip(sd / (3 * s), -1.0, 1.0).astype(np.float32)
    W = np.ones_like(F, np.uint8)
    W[:, :, : n // 8] = 0  # an unobserved slab
    C = ((np.arange((2 * n) ** 3, dtype=np.uint32) * 2654435761) & 0xFFFFFF).reshape((2 * n,) * 3) | (9 << 24)
    return F, W, C.astype(np.uint32), s


@pytest.mark.parametrize("kind", ["plane", "sphere"])
@pytest.mark.parametrize("device", [False, True])
def test_analytic_volumes(kind, device):
    F, W, C, s = analytic(kind)
    n = F.shape[0]
    vol = T.Volume((n,) * 3, (2 * n,) * 3, s, 3 * s, 64)
    vol.write(F, W, C)
    K = synth.intrinsics(150.0, 150.0, 79.5, 59.5)
    Tc = synth.look_at((0.35, -0.25, 0.4), (0.0, 0.0, -0.05))
    size, near, far, sf, sn = (160, 120), 0.05, 2.0, np.float32(1.5 * s), np.float32(0.5 * s)
    g = vol.raycast(K, Tc, size, near, far, float(sf), float(sn), device="cuda" if device else None)
    if device:
        g = {k: v.cpu().numpy() for k, v in g.items()}
    o = oracle.raycast(F, W, C, s, s / 2, vol.info().origin, K, Tc, size, near, far, float(sf), float(sn))
    exact = assert_same(g, o, kind)
    assert o["hits"] > 5000 and (o["range"] == 0).sum() > 100
    assert exact == 1.0
    vol.close()


def test_oracle_fused_sequence_from_a_view():
    """Volumes fused by the oracle from a synthetic sequence (noisy depth,
    partial observation), cast from one of its cameras."""
    seq = synth.sequence_small(n_frames=4, dims_geo=64, seed=3)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=8)
    for f in range(4):
        d, c = seq.frame(f)
        o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    vol.write(o.F, o.W, o.C)
    size = (320, 240)
    K = synth.intrinsics(262.5, 262.5, 159.5, 119.5)
    for f in (0, 2):
        g = vol.raycast(K, seq.poses[f], size, 0.1, 3.0)
        info = vol.info()
        r = oracle.raycast(o.F, o.W, o.C, seq.voxel_size, info.voxel_col, info.origin, K, seq.poses[f], size, 0.1,
                           3.0, step_far=float(np.float32(0.5 * np.float64(np.float32(seq.mu)))),
                           step_near=float(np.float32(0.5 * np.float64(np.float32(seq.voxel_size)))))
        assert_same(g, r, "frame %d" % f)
        assert r["hits"] > 0.3 * size[0] * size[1]
        assert ((r["rgbw"] >> 24) > 0).sum() > 0.2 * r["hits"]
    vol.close()


def test_raycast_rejects_bad_arguments():
    vol = T.Volume((16,) * 3, (16,) * 3, 1 / 16, 3 / 16, 8)
    K = synth.intrinsics(100.0, 100.0, 31.5, 23.5)
    good = synth.look_at((0.0, 0.3, 1.0), (0.0, 0.0, 0.0))
    vol.raycast(K, good, (64, 48))  # valid arguments are accepted
    bad = good.copy()
    bad[:3, 0] *= 2.0
    for args in [dict(near=1.0, far=0.5), dict(near=-0.1), dict(far=2000.0), dict(step_near=1e-9),
                 dict(step_far=0.001, step_near=0.01)]:
        with pytest.raises(T.TsdfError) as e:
            vol.raycast(K, good, (64, 48), **args)
        assert e.value.status == T.TSDF_ERR_INVALID_ARG
    with pytest.raises(T.TsdfError):
        vol.raycast(K, bad, (64, 48))
    with pytest.raises(T.TsdfError):
        vol.raycast(np.zeros((3, 3)), good, (64, 48))
    with pytest.raises(T.TsdfError):
        vol.raycast(K, good, (0, 48))
    vol.close()
