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


def run_batch(data, blocks=None, graph=True, tile=1):
    vols = make_volumes(data)
    b = T.Batch(vols)
    if blocks is not None:
        b.set_schedule(blocks, graph, tile)
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


@pytest.mark.parametrize("blocks,graph,tile", [(1, True, 1), (2, False, 4), (3, True, 8), (2, True, 2)])
def test_schedule_does_not_change_results(data, reference, blocks, graph, tile):
    out, _ = run_batch(data, blocks, graph, tile)
    for (a, r) in zip(out, reference):
        for x, y in zip(a, r):
            np.testing.assert_array_equal(x, y)


def test_autotune_keeps_a_valid_schedule_and_leaves_volumes_alone(data):
    vols = make_volumes(data)
    b = T.Batch(vols)
    before = [v.read() for v in vols]
    (best, tile), ms = b.autotune([frames[0] for _, frames in data], rounds=2)
    x, mx, t, g = b.schedule()
    assert 1 <= best <= mx and x == best and t == tile and tile in (1, 2, 4, 8)
    assert len(ms) == 4 * mx and all(m > 0 for m in ms)
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


def test_batched_equals_the_oracle_at_scan_sizes():
    """Scans of the 64-scan batched workload itself (720p RGB, 2x colour),
    including its largest (368^3 / 736^3) and smallest (64^3 / 128^3) edges,
    integrated in one batched launch per step and compared with the oracle
    over the whole volumes: weights and colours bit for bit, TSDF within 1e-5."""
    import os

    import oracle

    edges = synth.batched_edges(64)
    order = np.argsort(edges)
    pick = [int(order[-1]), int(order[0]), int(order[len(order) // 4]), int(order[len(order) // 2]),
            int(order[3 * len(order) // 4]), int(order[-2])]
    n_frames = 3
    data = []
    for i in pick:
        seq = synth.sequence_batched_scan(i, n_frames=n_frames)
        frames = []
        for f in range(n_frames):
            d, c = seq.frame(f)
            frames.append((d, c))
        data.append((seq, frames))
    assert max(s.dims_geo[0] for s, _ in data) == max(edges) and min(s.dims_geo[0] for s, _ in data) == min(edges)
    vols = [T.Volume(s.dims_geo, s.dims_col, s.voxel_size, s.mu, s.max_weight) for s, _ in data]
    b = T.Batch(vols)
    for f in range(n_frames):
        b.integrate([(torch.from_numpy(fr[f][0].view(np.int16)).cuda(), torch.from_numpy(fr[f][1]).cuda(),
                      s.K_depth, s.K_rgb, s.poses[f], s.T_depth_rgb) for s, fr in data])
    b.synchronize()
    nt = os.cpu_count() or 1
    for (s, fr), v in zip(data, vols):
        o = oracle.Oracle(s.dims_geo, s.dims_col, s.voxel_size, s.mu, s.max_weight, n_threads=nt)
        for f in range(n_frames):
            o.integrate(fr[f][0], fr[f][1], s.K_depth, s.K_rgb, s.poses[f], s.T_depth_rgb)
        F, W, C = v.read()
        np.testing.assert_array_equal(W, o.W, err_msg="weights, edge %d" % s.dims_geo[0])
        np.testing.assert_array_equal(C, o.C, err_msg="colours, edge %d" % s.dims_geo[0])
        assert float(np.abs(F - o.F).max()) <= 1e-5
        assert (W > 0).sum() > 1000 and ((C >> 24) > 0).sum() > 100
    b.close()
    for v in vols:
        v.close()
