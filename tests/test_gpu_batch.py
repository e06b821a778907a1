"""Batched fusion (one persistent, graph-captured launch per step for many
scans of uneven sizes) against per-scan tsdf_integrate: identical volumes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1602_06645_gb300 as T  # noqa: E402
from paper_1602_06645_gb300 import synth  # noqa: E402

EDGES = [16, 40, 24, 56, 32, 48, 8, 64]


def scans(n_frames=3, edges=EDGES):
    out = []
    for i, e in enumerate(edges):
        seq = synth.sequence_batched_scan(i, n_frames=n_frames, edge=e)
        seq.rgb_size = (320, 180)
        seq.K_rgb = synth.intrinsics(175.0, 175.0, 159.5, 89.5)
        frames = []
        for f in range(n_frames):
            d, c = seq.frame(f)
            frames.append((torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda(), seq.K_depth,
                           seq.K_rgb, seq.poses[f], seq.T_depth_rgb))
        out.append((seq, frames))
    return out


def make_volumes(data):
    return [T.Volume(s.dims_geo, s.dims_col, s.voxel_size, s.mu, s.max_weight) for s, _ in data]


@pytest.fixture(scope="module")
def data():
    return scans()


@pytest.fixture(scope="module")
def reference(data):
    vols = make_volumes(data)
    for v, (s, frames) in zip(vols, data):
        for fr in frames:
            v.integrate(*fr)
    out = [v.read() for v in vols]
    for v in vols:
        v.close()
    return out


def run_batch(data, blocks=None, graph=True):
    vols = make_volumes(data)
    b = T.Batch(vols)
    if blocks is not None:
        b.set_schedule(blocks, graph)
    for f in range(len(data[0][1])):
        b.integrate([frames[f] for _, frames in data])
    b.synchronize()
    out = [v.read() for v in vols]
    stats = [v.stats() for v in vols]
    b.close()
    for v in vols:
        v.close()
    return out, stats


def test_batched_equals_sequential(data, reference):
    out, stats = run_batch(data)
    for (a, r) in zip(out, reference):
        for x, y in zip(a, r):
            np.testing.assert_array_equal(x, y)
    assert sum(s.total_col_updated for s in stats) > 1000


@pytest.mark.parametrize("blocks,graph", [(1, True), (2, False), (3, True)])
def test_schedule_does_not_change_results(data, reference, blocks, graph):
    out, _ = run_batch(data, blocks, graph)
    for (a, r) in zip(out, reference):
        for x, y in zip(a, r):
            np.testing.assert_array_equal(x, y)


def test_autotune_keeps_a_valid_schedule_and_leaves_volumes_alone(data):
    vols = make_volumes(data)
    b = T.Batch(vols)
    before = [v.read() for v in vols]
    best, ms = b.autotune([frames[0] for _, frames in data], rounds=2)
    x, mx, g = b.schedule()
    assert 1 <= best <= mx and x == best and len(ms) == mx and all(m > 0 for m in ms)
    after = [v.read() for v in vols]
    for p, q in zip(before, after):
        for x1, y1 in zip(p, q):
            np.testing.assert_array_equal(x1, y1)
    b.close()
    for v in vols:
        v.close()


def test_stalled_barrier_times_out_and_the_batch_recovers(data, reference):
    """A block that never arrives at the first grid barrier makes the other
    blocks' bounded waits run out: the host sees TSDF_ERR_TIMEOUT, and the
    context and the batch stay usable."""
    vols = make_volumes(data)
    b = T.Batch(vols)
    T.tsdf_batch_inject_stall(b.b)
    b.integrate([frames[0] for _, frames in data])
    with pytest.raises(T.TsdfError) as e:
        b.synchronize()
    assert e.value.status == T.TSDF_ERR_TIMEOUT
    b.close()
    for v in vols:
        v.close()
    out, _ = run_batch(data)  # fresh volumes: still exact
    for (a, r) in zip(out, reference):
        for x, y in zip(a, r):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("edge", [48, 44])
def test_one_scan_in_one_launch_equals_plain(edge):
    """A batch of one volume is the single-launch fused form of the frame
    (geometry, band gate and colour in one persistent launch with grid
    barriers): same volumes as the six-kernel path."""
    one = scans(n_frames=4, edges=[edge])
    vol = make_volumes(one)[0]
    for fr in one[0][1]:
        vol.integrate(*fr)
    ref = vol.read()
    vol.close()
    out, stats = run_batch(one)
    for a, b in zip(ref, out[0]):
        np.testing.assert_array_equal(a, b)
    assert stats[0].total_col_updated > 100
