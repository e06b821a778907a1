"""GPU mesh extraction (marching cubes, and marching tetrahedra as an option)
and texture maps against the oracle (mesh.c).

Volumes come from outside the CUDA path (analytic signed distances, or the
oracle's own fusion of a synthetic sequence) and are written into the GPU
volume.  The GPU returns triangles in no fixed order, so triangle sets are
compared (each triangle bit for bit); texture layouts and texels must match
bit for bit.
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


def tri_set(tris):
    a = np.ascontiguousarray(np.asarray(tris, np.float32).reshape(-1, 9)).view(np.uint32)
    return a[np.lexsort(a.T[::-1])]


def sphere_volume(n):
    s = 1.0 / n
    c = -0.5 + (np.arange(n, dtype=np.float64) + 0.5) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    sd = np.sqrt((x - 0.031) ** 2 + (y + 0.022) ** 2 + (z - 0.017) ** 2) - 0.29
    F = np.clip(sd / (3 * s), -1.0, 1.0).astype(np.float32)
    W = np.ones_like(F, np.uint8)
    W[: n // 5] = 0  # an unobserved slab: cells touching it give nothing
    return F, W, s


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
@pytest.mark.parametrize("n", [40, 45])  # whole bricks, and ragged bricks at the + faces
def test_analytic_sphere_mesh_equals_oracle(n, method):
    F, W, s = sphere_volume(n)
    vol = T.Volume((n,) * 3, (n,) * 3, s, 3 * s, 64)
    vol.write(F, W)
    g = vol.mesh(method=method)
    o = oracle.mesh(F, W, s, vol.info().origin, method)
    assert len(o) > 1000
    np.testing.assert_array_equal(tri_set(g), tri_set(o))
    # device output, and a buffer too small: the count is still the total
    gd = vol.mesh(device="cuda", method=method).cpu().numpy()
    np.testing.assert_array_equal(tri_set(gd), tri_set(o))
    part = np.zeros((100, 3, 3), np.float32)
    assert T.tsdf_mesh_ex(vol.h, {"cubes": 0, "tetrahedra": 1}[method], part, 100) == len(o)
    full = set(map(bytes, tri_set(o)))
    assert all(bytes(t) in full for t in tri_set(part))
    vol.close()


@pytest.fixture(scope="module")
def fused():
    seq = synth.sequence_small(n_frames=4, dims_geo=64, seed=3)
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=8)
    for f in range(4):
        d, c = seq.frame(f)
        o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    vol.write(o.F, o.W, o.C)
    yield seq, o, vol
    vol.close()


@pytest.mark.parametrize("method", ["cubes", "tetrahedra"])
def test_fused_sequence_mesh_equals_oracle(fused, method):
    seq, o, vol = fused
    ref = oracle.mesh(o.F, o.W, seq.voxel_size, vol.info().origin, method)
    assert len(ref) > 5000
    np.testing.assert_array_equal(tri_set(vol.mesh(method=method)), tri_set(ref))


@pytest.mark.parametrize("seed", range(3))
def test_random_fields_mesh_equals_oracle(seed):
    """Random corner values everywhere (every marching-cubes case, many
    ambiguous faces), ragged volume: triangle sets equal bit for bit."""
    rng = np.random.default_rng(seed)
    dims = (37, 29, 21)
    F = rng.uniform(-1, 1, size=dims[::-1]).astype(np.float32)
    W = (rng.uniform(size=dims[::-1]) > 0.02).astype(np.uint8)
    vol = T.Volume(dims, dims, 0.01, 0.03, 64)
    vol.write(F, W)
    o = oracle.mesh(F, W, 0.01, vol.info().origin, "cubes")
    assert len(o) > 20000
    np.testing.assert_array_equal(tri_set(vol.mesh()), tri_set(o))
    vol.close()


@pytest.mark.parametrize("device", [False, True])
def test_texture_maps_equal_oracle(fused, device):
    seq, o, vol = fused
    info = vol.info()
    tris = oracle.mesh(o.F, o.W, seq.voxel_size, info.origin)[::7].copy()
    size = float(info.voxel_col) * 0.5
    wh_o, off_o, tex_o = oracle.texture_maps(tris, o.C, info.voxel_col, info.origin, size)
    arg = torch.from_numpy(tris).cuda() if device else tris
    wh, off, tex = vol.texture_maps(arg, size)
    if device:
        wh, off, tex = wh.cpu().numpy(), off.cpu().numpy(), tex.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(wh, wh_o)
    np.testing.assert_array_equal(off, off_o)
    np.testing.assert_array_equal(tex, tex_o)
    assert ((tex_o >> 24) == 255).mean() > 0.5


def test_mesh_and_texture_arguments_are_checked(fused):
    _, _, vol = fused
    with pytest.raises(T.TsdfError):
        T.tsdf_mesh(vol.h, None, 10)
    tri = np.zeros((1, 3, 3), np.float32)
    with pytest.raises(T.TsdfError):
        vol.texture_maps(tri, 0.0)
    with pytest.raises(T.TsdfError):
        vol.texture_maps(tri, 0.01, max_side=1)
