"""z-slab handles on one GPU against a whole-volume handle: the slabs' own
parts (read_slab), concatenated in z order, equal the whole volume bit for bit
(geometry, weights and colours), for two and three slabs, colour/geometry
ratios 1, 2 and 5/3, the plain path and the batched launch; a slab's
checkpoint round-trips.  The same partition is checked against the oracle
over gloo ranks on the CPU (tests/test_slabs_multirank.py)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1602_06645_gb300 as T  # noqa: E402
from paper_1602_06645_gb300 import synth  # noqa: E402


def _frames(seq, n):
    out = []
    for f in range(n):
        d, c = seq.frame(f)
        out.append((torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda(), seq.K_depth, seq.K_rgb,
                    seq.poses[f], seq.T_depth_rgb))
    return out


def _seq(dims_geo, dims_col):
    seq = synth.sequence_small(n_frames=4, dims_geo=dims_geo)
    seq.dims_col = (dims_col,) * 3
    return seq


@pytest.mark.parametrize("dims_geo,dims_col,n,schedule", [
    (48, 96, 2, "kernels"), (48, 96, 3, "kernels"), (64, 64, 2, "kernels"), (48, 80, 2, "kernels"),
    (40, 80, 3, "kernels"), (48, 96, 3, "fused"), (40, 80, 2, "fused")])
def test_slabs_equal_the_whole_volume(dims_geo, dims_col, n, schedule):
    """Slab handles (either frame schedule) against a whole-volume handle run
    as the kernel chain."""
    seq = _seq(dims_geo, dims_col)
    frames = _frames(seq, 4)
    args = (seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    whole = T.Volume(*args)
    sched = T.TSDF_SCHEDULE_FUSED if schedule == "fused" else T.TSDF_SCHEDULE_KERNELS
    slabs = [T.Volume(*args, slab=r, schedule=sched) for r in T.slab_ranges(seq.dims_geo, seq.dims_col, n)]
    for fr in frames:
        whole.integrate(*fr)
        for v in slabs:
            v.integrate(*fr)
    F, W, C = whole.read()
    parts = [v.read_slab() for v in slabs]
    np.testing.assert_array_equal(np.concatenate([p[0] for p in parts]).view(np.uint32), F.view(np.uint32))
    np.testing.assert_array_equal(np.concatenate([p[1] for p in parts]), W)
    np.testing.assert_array_equal(np.concatenate([p[2] for p in parts]), C)
    assert (W > 0).sum() > 5000 and ((C >> 24) > 0).sum() > 1000
    for v in slabs + [whole]:
        v.close()


def test_batched_slabs_equal_the_whole_volume():
    seq = _seq(48, 96)
    frames = _frames(seq, 3)
    args = (seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    whole = T.Volume(*args)
    for fr in frames:
        whole.integrate(*fr)
    slabs = [T.Volume(*args, slab=r) for r in T.slab_ranges(seq.dims_geo, seq.dims_col, 2)]
    b = T.Batch(slabs)
    for fr in frames:
        b.integrate([fr, fr])
    b.synchronize()
    F, W, C = whole.read()
    parts = [v.read_slab() for v in slabs]
    np.testing.assert_array_equal(np.concatenate([p[1] for p in parts]), W)
    np.testing.assert_array_equal(np.concatenate([p[2] for p in parts]), C)
    np.testing.assert_array_equal(np.concatenate([p[0] for p in parts]).view(np.uint32), F.view(np.uint32))
    b.close()
    for v in slabs + [whole]:
        v.close()


def test_slab_checkpoint_round_trip_and_whole_volume_only_calls(tmp_path):
    seq = _seq(48, 96)
    frames = _frames(seq, 3)
    args = (seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    a = T.Volume(*args, slab=(24, 48))
    for fr in frames[:2]:
        a.integrate(*fr)
    path = str(tmp_path / "slab.tsdf")
    T.tsdf_save(a.h, path)
    b = T.Volume(*args, slab=(24, 48))
    T.tsdf_load(b.h, path)
    for v in (a, b):
        v.integrate(*frames[2])
    for x, y in zip(a.read(), b.read()):
        np.testing.assert_array_equal(x, y)
    other = T.Volume(*args, slab=(0, 24))
    with pytest.raises(T.TsdfError):
        T.tsdf_load(other.h, path)  # another slab's checkpoint
    with pytest.raises(T.TsdfError):
        a.raycast(seq.K_depth, seq.poses[0], (64, 48))
    with pytest.raises(T.TsdfError):
        T.Volume(*args, slab=(24, 49))
    info = T.tsdf_get_info(a.h)
    assert tuple(info.held_geo_z) == (23, 48) and tuple(info.held_col_z) == (48, 96) and info.dims_geo[2] == 48
    for v in (a, b, other):
        v.close()
