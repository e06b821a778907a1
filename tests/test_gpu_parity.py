"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Weights and 8-bit colours must match bit for bit, the TSDF within 1e-5 in
normalised units (the binary32 operation order is shared, so it is expected
to match exactly as well).  Inputs are the seeded synthetic sequences and
random frames; sizes span many bricks with ragged tails.
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

NT = os.cpu_count() or 1
F_TOL = 1e-5


def assert_parity(o, F, W, C, label=""):
    np.testing.assert_array_equal(W, o.W, err_msg="geometry weights " + label)
    dF = np.abs(F - o.F)
    assert dF.max() <= F_TOL, "TSDF differs by %g %s" % (dF.max(), label)
    bad = np.nonzero(C != o.C)
    assert bad[0].size == 0, "colour voxels differ at %d places, first %s: gpu %08x oracle %08x %s" % (
        bad[0].size, tuple(int(b[0]) for b in bad), int(C[bad][0]), int(o.C[bad][0]), label)


def run_sequence(seq, frames, okw=None, vkw=None, device_inputs=False):
    okw = dict(okw or {})
    vkw = dict(vkw or {})
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, n_threads=NT, **okw)
    v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, **okw, **vkw)
    counts = []
    for f in frames:
        d, c = seq.frame(f)
        n_orc = o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        if device_inputs:
            d, c = torch.from_numpy(d.astype(np.int16).view(np.uint16).copy()).cuda(), torch.from_numpy(c).cuda()
        v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        st = v.stats()
        counts.append((n_orc, (st.geo_updated, st.col_updated)))
    F, W, C = v.read()
    v.close()
    return o, F, W, C, counts


@pytest.fixture(scope="module")
def small_run():
    seq = synth.sequence_small(n_frames=10)
    return seq, run_sequence(seq, range(10))


def test_small_sequence_full_volume_parity(small_run):
    """128^3 geometry / 256^3 colour, 10 frames: every voxel of both volumes."""
    seq, (o, F, W, C, counts) = small_run
    assert_parity(o, F, W, C)
    assert (W > 0).sum() > 100000 and ((C >> 24) > 0).sum() > 50000
    assert np.array_equal(F, o.F), "TSDF not bit-identical (max diff %g)" % np.abs(F - o.F).max()


def test_small_sequence_update_counts(small_run):
    """The per-frame updated-voxel counters equal the oracle's counts."""
    _, (_, _, _, _, counts) = small_run
    for orc, gpu in counts:
        assert tuple(orc) == tuple(gpu)


def test_culling_changes_nothing():
    """Dense sweep (culling off) and culled runs give identical volumes."""
    seq = synth.sequence_small(n_frames=4, dims_geo=64, seed=11)
    outs = []
    for cull in (True, False):
        v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, culling=cull)
        for f in range(4):
            d, c = seq.frame(f)
            v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        outs.append(v.read())
        v.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims_geo,dims_col", [
    ((40, 24, 36), (40, 24, 36)),      # ratio 1, ragged bricks
    ((36, 28, 20), (108, 84, 60)),     # ratio 3
    ((24, 24, 24), (40, 40, 40)),      # ratio 5/3 (non-integer)
    ((20, 12, 28), (40, 24, 56)),      # ratio 2, dims not multiples of 8
    ((12, 8, 12), (96, 64, 96)),       # ratio 8, the largest supported: over 32 owned indices per axis
])
def test_ratios_and_ragged_dims(dims_geo, dims_col):
    seq = synth.sequence_small(n_frames=4, seed=5)
    seq.dims_geo, seq.dims_col = dims_geo, dims_col
    seq.voxel_size = float(np.float32(0.9 / dims_geo[0]))
    seq.mu = float(np.float32(3 * seq.voxel_size))
    o, F, W, C, _ = run_sequence(seq, range(4))
    assert_parity(o, F, W, C, str(dims_col))
    assert ((C >> 24) > 0).sum() > 100


@pytest.mark.parametrize("mode", ["bilinear", "paper_normal", "no_free_space", "max_weight_2", "wide_band"])
def test_modes(mode):
    seq = synth.sequence_small(n_frames=5, dims_geo=48, seed=7)
    okw = {"bilinear": dict(sample_mode=1), "paper_normal": dict(colour_mode=1),
           "no_free_space": dict(update_free_space=0), "max_weight_2": {}, "wide_band": dict(band=0.9, sigma=0.05)}[mode]
    if mode == "max_weight_2":
        seq.max_weight = 2
    o, F, W, C, _ = run_sequence(seq, range(5), okw)
    assert_parity(o, F, W, C, mode)


def test_record_buffer_overflow_path_is_exact(monkeypatch):
    """With a voxel-record buffer of 5 entries almost every band-passing voxel
    is finished by the band kernel itself; the volumes still equal the
    oracle's."""
    monkeypatch.setenv("TSDF_VOXEL_RECORD_CAPACITY", "5")
    seq = synth.sequence_small(n_frames=4, dims_geo=64, seed=17)
    o, F, W, C, _ = run_sequence(seq, range(4))
    assert_parity(o, F, W, C, "overflow")
    assert ((C >> 24) > 0).sum() > 1000


def test_device_and_host_inputs_agree():
    seq = synth.sequence_small(n_frames=3, dims_geo=48, seed=9)
    o1, F1, W1, C1, _ = run_sequence(seq, range(3))
    o2, F2, W2, C2, _ = run_sequence(seq, range(3), device_inputs=True)
    np.testing.assert_array_equal(F1, F2)
    np.testing.assert_array_equal(W1, W2)
    np.testing.assert_array_equal(C1, C2)


def random_frames(rng, n, W=48, H=36, cW=96, cH=72):
    from test_oracle_pins import K_of, plane_depth_image
    Kd, Kr = K_of(50.0, W, H), K_of(90.0, cW, cH)
    out = []
    for f in range(n):
        az, el = rng.uniform(0, 2 * np.pi), rng.uniform(-0.7, 0.7)
        dist = rng.uniform(0.45, 0.9)
        pos = dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        Twd = synth.look_at(pos, rng.normal(size=3) * 0.05).astype(np.float32)
        base = plane_depth_image(Kd, W, H, dist + rng.uniform(-0.08, 0.08), rng.uniform(-0.4, 0.4),
                                 rng.uniform(-0.4, 0.4)).astype(np.int64)
        depth = np.clip(base + rng.integers(-20, 21, size=base.shape), 0, 65535).astype(np.uint16)
        depth[rng.random(depth.shape) < 0.05] = 0
        rgb = rng.integers(0, 256, size=(cH, cW, 3), dtype=np.uint8)
        out.append((depth, rgb, Kd, Kr, Twd))
    return out


@pytest.mark.parametrize("seed", range(12))
def test_random_frames_small_volumes(seed):
    """Random poses, depths and colours on 8^3..24^3 volumes (several bricks,
    ragged tails): bit-exact weights and colours, exact TSDF."""
    rng = np.random.default_rng(seed)
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
    v = T.Volume(gd, cd, s, mu, mw, **kw)
    for depth, rgb, Kd, Kr, Twd in random_frames(rng, 5):
        o.integrate(depth, rgb, Kd, Kr, Twd, Tdr)
        v.integrate(depth, rgb, Kd, Kr, Twd, Tdr)
    F, W, C = v.read()
    v.close()
    assert_parity(o, F, W, C, "seed %d" % seed)
    assert np.array_equal(F, o.F)


def test_empty_frame_changes_nothing():
    """An all-invalid depth image (every pixel 0) updates no voxel."""
    seq = synth.sequence_small(n_frames=2, dims_geo=32)
    v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
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


def test_read_write_roundtrip_and_resume(tmp_path):
    """integrate 6 == integrate 3 -> save -> load into a new handle -> integrate 3."""
    seq = synth.sequence_small(n_frames=6, dims_geo=40, seed=13)
    frames = [seq.frame(f) for f in range(6)]
    args = (seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    a = T.Volume(*args)
    for f, (d, c) in enumerate(frames):
        a.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    ref = a.read()
    a.close()
    b = T.Volume(*args)
    for f, (d, c) in enumerate(frames[:3]):
        b.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    path = tmp_path / "ckpt.tsdf"
    b.save(path)
    b.close()
    c2 = T.Volume(*args)
    c2.load(path)
    assert c2.info().frames == 3
    for f, (d, c) in enumerate(frames[3:], start=3):
        c2.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    got = c2.read()
    # device-pointer read agrees with the host read
    Fd, Wd, Cd = c2.read_torch()
    c2.close()
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(Fd.cpu().numpy(), got[0])
    np.testing.assert_array_equal(Wd.cpu().numpy(), got[1])
    np.testing.assert_array_equal(Cd.cpu().numpy().view(np.uint32), got[2])


def test_invalid_frame_arguments_are_rejected():
    seq = synth.sequence_small(n_frames=1, dims_geo=16)
    v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    d, c = seq.frame(0)
    bad_T = seq.poses[0].copy()
    bad_T[:3, 0] *= 1.1  # not a rotation (column norm 1.1)
    for args in [(d, c, seq.K_depth, seq.K_rgb, bad_T, seq.T_depth_rgb),
                 (d, c, np.zeros((3, 3)), seq.K_rgb, seq.poses[0], seq.T_depth_rgb),
                 (d, c, seq.K_depth, seq.K_rgb, np.full((4, 4), np.nan), seq.T_depth_rgb)]:
        with pytest.raises(T.TsdfError) as e:
            v.integrate(*args)
        assert e.value.status == T.TSDF_ERR_INVALID_ARG
    v.close()


def test_phase_profile_and_phase_mask():
    """Phase timing sees every phase of a frame; with a mask only the chosen
    phase is timed, and the volumes do not depend on either."""
    seq = synth.sequence_small(n_frames=3, dims_geo=48, seed=9)
    vols = [T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight) for _ in range(2)]
    vols[0].profile(True)
    vols[1].profile(True)
    vols[1].profile_phases(["geometry"])
    for f in range(3):
        d, c = seq.frame(f)
        for v in vols:
            v.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    full, n_full = vols[0].profile_read()
    one, n_one = vols[1].profile_read()
    assert n_full == n_one == 3
    assert all(full[k] > 0 for k in T.PHASES)
    assert one["geometry"] > 0 and all(one[k] == 0 for k in T.PHASES if k != "geometry")
    for a, b in zip(vols[0].read(), vols[1].read()):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(T.TsdfError):
        T.tsdf_profile_phases(vols[0].h, 0)
    for v in vols:
        v.close()


STAT_FIELDS = [f for f, _ in T.tsdf_stats._fields_]


@pytest.mark.parametrize("device_inputs,profiled", [(False, False), (True, False), (False, True)])
def test_async_stats_equal_synchronous_reads(device_inputs, profiled):
    """Counters read with tsdf_stats_request / tsdf_stats_collect while the
    next frame is already queued equal those of a synchronous read after each
    frame, field by field.  The next frame's depth tiles reset the
    geometry-side counters: after a pipelined frame those are read from a
    copy queued ahead of them, and with the first phases timed (no
    pipelining) the depth tiles wait for the single copy."""
    seq = synth.sequence_small(n_frames=12)
    frames = []
    for f in range(12):
        d, c = seq.frame(f)
        if device_inputs:
            d, c = torch.from_numpy(d.view(np.int16).copy()).cuda(), torch.from_numpy(c).cuda()
        frames.append((d, c))
    args = lambda f: (*frames[f], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    a = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    sync = []
    for f in range(12):
        a.integrate(*args(f))
        sync.append(a.stats())
    b = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    if profiled:
        b.profile(True)
    assert all(getattr(b.stats_collect(1), k) == 0 for k in STAT_FIELDS if k != "total_bricks")  # never requested
    got = []
    for f in range(12):
        b.integrate(*args(f))
        b.stats_request(f & 1)
        if f:
            got.append(b.stats_collect((f - 1) & 1))
    got.append(b.stats_collect(11 & 1))
    for f, (x, y) in enumerate(zip(sync, got)):
        for k in STAT_FIELDS:
            assert getattr(x, k) == getattr(y, k), (f, k, getattr(x, k), getattr(y, k))
    assert sync[-1].frames_counted == 12 and sync[-1].geo_updated > 0
    for bad in (-1, 2):
        with pytest.raises(T.TsdfError):
            b.stats_request(bad)
        with pytest.raises(T.TsdfError):
            b.stats_collect(bad)
    Fa, Wa, Ca = a.read()
    Fb, Wb, Cb = b.read()
    a.close()
    b.close()
    assert np.array_equal(Fa, Fb) and np.array_equal(Wa, Wb) and np.array_equal(Ca, Cb)


def test_device_depth_written_on_the_handle_stream_just_before_the_call():
    """A device depth image written by work queued on the handle's stream
    right before tsdf_integrate (behind a GPU sleep, so the write is late) is
    read only after that work: the volumes equal those of the same frames
    passed as ready device images.  With the inputs declared ready the
    second stream may start early, so such a caller must not declare it."""
    seq = synth.sequence_small(n_frames=4, dims_geo=48, seed=31)
    args = (seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight)
    frames = [seq.frame(f) for f in range(4)]
    ref = T.Volume(*args)
    for f, (d, c) in enumerate(frames):
        ref.integrate(torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda(), seq.K_depth,
                      seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    expected = ref.read()
    ref.close()
    v = T.Volume(*args)
    depth = torch.zeros(frames[0][0].shape, dtype=torch.int16, device="cuda")
    for f, (d, c) in enumerate(frames):
        # both uploads before the sleep: a pageable upload after it would make
        # the host wait for the stream, and the write would no longer be late
        src = torch.from_numpy(d.view(np.int16)).cuda()
        rgb = torch.from_numpy(c).cuda()
        torch.cuda.synchronize()
        torch.cuda._sleep(20_000_000)  # ~10 ms on the handle's stream before the write
        depth.copy_(src)
        v.integrate(depth, rgb, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    got = v.read()
    v.close()
    for a, b in zip(got, expected):
        np.testing.assert_array_equal(a, b)
