"""The fused frame schedule (TSDF_SCHEDULE_FUSED: geometry update, colour
candidates and band gate in one persistent launch) against the CPU oracle and
against the kernel chain: the same volumes bit for bit and the same counters,
over the small sequence, ragged dims and colour / geometry ratios, every
mode, random frames, the record-overflow path, an empty frame and the scan
workload; and its bounded wait, made to run out on purpose, reports
TSDF_ERR_TIMEOUT and the next frames run normally.
"""
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
from test_gpu_parity import assert_parity, random_frames  # noqa: E402

NT = os.cpu_count() or 1
FUSED = dict(schedule=T.TSDF_SCHEDULE_FUSED)
STAT_FIELDS = ("geo_updated", "col_updated", "geo_bricks", "col_bricks", "visible_bricks", "total_geo_updated",
               "total_col_updated", "total_col_bricks", "total_cells", "total_col_active_bricks",
               "total_geo_changed_bricks")


def run(seq, frames, okw=None, vkw=None, oracle_too=True):
    okw = dict(okw or {})
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=NT,
                      **okw) if oracle_too else None
    v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **okw, **(vkw or {}))
    counts, stats = [], []
    for f in frames:
        d, c = seq.frame(f)
        n_orc = o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb) if o else None
        v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        st = v.stats()
        counts.append((n_orc, (st.geo_updated, st.col_updated)))
        stats.append(tuple(getattr(st, k) for k in STAT_FIELDS))
    F, W, C = v.read()
    v.close()
    return o, F, W, C, counts, stats


def test_schedule_is_set_and_checked():
    v = T.Volume((16, 16, 16), (32, 32, 32), 0.01, 0.03, 8)
    assert v.schedule == T.TSDF_SCHEDULE_KERNELS
    v.schedule = T.TSDF_SCHEDULE_FUSED
    assert v.schedule == T.TSDF_SCHEDULE_FUSED
    with pytest.raises(T.TsdfError):
        v.schedule = 7
    v.close()


def test_small_sequence_equals_the_oracle_and_the_kernel_chain():
    """128^3 / 256^3, 10 frames: every voxel equals the oracle's; every
    per-frame counter equals the kernel chain's."""
    seq = synth.sequence_small(n_frames=10)
    o, F, W, C, counts, stats = run(seq, range(10), vkw=FUSED)
    assert_parity(o, F, W, C, "fused")
    assert np.array_equal(F, o.F)
    for orc, gpu in counts:
        assert tuple(orc) == tuple(gpu)
    _, F2, W2, C2, _, stats2 = run(seq, range(10), oracle_too=False)
    np.testing.assert_array_equal(F, F2)
    np.testing.assert_array_equal(W, W2)
    np.testing.assert_array_equal(C, C2)
    assert stats == stats2


@pytest.mark.parametrize("dims_geo,dims_col", [
    ((40, 24, 36), (40, 24, 36)),      # ratio 1, ragged bricks
    ((36, 28, 20), (108, 84, 60)),     # ratio 3
    ((24, 24, 24), (40, 40, 40)),      # ratio 5/3
    ((20, 12, 28), (40, 24, 56)),      # ratio 2, dims not multiples of 8
])
def test_ratios_and_ragged_dims(dims_geo, dims_col):
    seq = synth.sequence_small(n_frames=4, seed=5)
    seq.dims_geo, seq.dims_col = dims_geo, dims_col
    seq.voxel_size = float(np.float32(0.9 / dims_geo[0]))
    seq.mu = float(np.float32(3 * seq.voxel_size))
    o, F, W, C, _, _ = run(seq, range(4), vkw=FUSED)
    assert_parity(o, F, W, C, "fused " + str(dims_col))


@pytest.mark.parametrize("mode", ["bilinear", "paper_normal", "no_free_space", "max_weight_2", "wide_band",
                                  "no_culling"])
def test_modes(mode):
    seq = synth.sequence_small(n_frames=5, dims_geo=48, seed=7)
    okw = {"bilinear": dict(sample_mode=1), "paper_normal": dict(colour_mode=1),
           "no_free_space": dict(update_free_space=0), "max_weight_2": {}, "wide_band": dict(band=0.9, sigma=0.05),
           "no_culling": {}}[mode]
    vkw = dict(FUSED, culling=False) if mode == "no_culling" else FUSED
    if mode == "max_weight_2":
        seq.max_weight = 2
    o, F, W, C, _, _ = run(seq, range(5), okw, vkw)
    assert_parity(o, F, W, C, "fused " + mode)


def test_record_buffer_overflow_path(monkeypatch):
    monkeypatch.setenv("TSDF_VOXEL_RECORD_CAPACITY", "5")
    seq = synth.sequence_small(n_frames=4, dims_geo=64, seed=17)
    o, F, W, C, _, _ = run(seq, range(4), vkw=FUSED)
    assert_parity(o, F, W, C, "fused overflow")


@pytest.mark.parametrize("seed", range(6))
def test_random_frames_small_volumes(seed):
    rng = np.random.default_rng(100 + seed)
    gd = tuple(int(v) for v in rng.integers(6, 25, size=3))
    r = int(rng.integers(1, 4))
    cd = tuple(v * r for v in gd)
    s = float(np.float32(0.4 / max(gd)))
    mu = float(np.float32(rng.uniform(2, 5) * s))
    Tdr = np.eye(4, dtype=np.float32)
    Tdr[:3, 3] = (-0.025, 0.003, 0.001)
    kw = dict(sample_mode=int(rng.integers(0, 2)), colour_mode=int(rng.integers(0, 2)), band=float(rng.uniform(0.2, 0.8)),
              sigma=float(rng.uniform(0.01, 0.05)), origin=(-0.2, -0.2, -0.2))
    mw = int(rng.integers(1, 6))
    o = oracle.Oracle(gd, cd, s, mu, mw, **kw)
    v = T.Volume(gd, cd, s, mu, mw, **kw, **FUSED)
    for depth, rgb, Kd, Kr, Twd in random_frames(rng, 5):
        o.integrate(depth, rgb, Kd, Kr, Twd, Tdr)
        v.integrate(depth, rgb, Kd, Kr, Twd, Tdr)
    F, W, C = v.read()
    v.close()
    assert_parity(o, F, W, C, "fused seed %d" % seed)
    assert np.array_equal(F, o.F)


def test_empty_frame_changes_nothing():
    seq = synth.sequence_small(n_frames=2, dims_geo=32)
    v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **FUSED)
    d, c = seq.frame(0)
    v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[0], seq.T_depth_rgb)
    before = v.read()
    v.integrate(np.zeros_like(d), c, seq.K_depth, seq.K_rgb, seq.poses[1], seq.T_depth_rgb)
    st = v.stats()
    after = v.read()
    v.close()
    assert st.geo_updated == 0 and st.col_updated == 0
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


def test_scan_workload_equals_the_kernel_chain():
    """512^3 / 1024^3 over 12 frames of the scan orbit, device frames, both
    schedules on the same frames: both volumes equal bit for bit (compared on
    the device) and so do the counters."""
    seq = synth.sequence_scan(n_frames=12)
    frames = []
    for f in range(12):
        d, c = seq.frame(f)
        frames.append((torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda()))
    outs, stats = [], []
    for sched in (T.TSDF_SCHEDULE_KERNELS, T.TSDF_SCHEDULE_FUSED):
        v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, schedule=sched)
        st = []
        for f, (d, c) in enumerate(frames):
            v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
            s = v.stats()
            st.append(tuple(getattr(s, k) for k in STAT_FIELDS))
        outs.append(v.read_torch())
        stats.append(st)
        v.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert stats[0] == stats[1]
    assert stats[1][-1][1] > 100000  # colour voxels updated in the last frame


def test_a_wait_that_runs_out_reports_timeout_and_the_next_frames_run():
    """One visible brick is never released (test injection): the wait for it
    gives up after 1 s, the synchronising call reports TSDF_ERR_TIMEOUT, the
    frame's geometry is still complete, and the following frames give the
    kernel chain's geometry and report no error."""
    seq = synth.sequence_small(n_frames=5, dims_geo=64, seed=3)
    vf = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **FUSED)
    vk = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    for f in range(5):
        d, c = seq.frame(f)
        if f == 2:
            T.tsdf_fused_inject_stall(vf.h)
        vf.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        vk.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        if f == 2:
            with pytest.raises(T.TsdfError) as err:
                T.tsdf_synchronize(vf.h)
            assert err.value.status == T.TSDF_ERR_TIMEOUT
        else:
            T.tsdf_synchronize(vf.h)
    Ff, Wf, _ = vf.read()
    Fk, Wk, _ = vk.read()
    vf.close()
    vk.close()
    np.testing.assert_array_equal(Wf, Wk)
    np.testing.assert_array_equal(Ff, Fk)
