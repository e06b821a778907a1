"""The allocation-free geometry entry point against the regular one and the
oracle.

tsdf_integrate_geometry_static is for callers that cannot allocate device
memory (another framework owns the allocator, or the device-memory budget is
fixed in advance): they pass their own TSDF and weight arrays and the library
uses a fixed scratch array compiled into it.  Its results must equal the
geometry volume that tsdf_integrate produces, call after call, and the
oracle's geometry update.
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

F_TOL = 1e-5  # the TSDF tolerance used by the parity tests


def _origin(dims, s):
    return tuple(float(np.float32(-0.5 * float(n) * float(s))) for n in dims)


@pytest.mark.parametrize("dims", [(96, 80, 72), (90, 70, 60)])
def test_static_entry_matches_regular_entry_two_calls(dims):
    seq = synth.sequence_small(n_frames=2, dims_geo=dims[0], seed=21)
    s = float(np.float32(1.0 / dims[0]))
    mu = float(np.float32(3 * s))
    mw = seq.max_weight
    vol = T.Volume(dims, dims, s, mu, mw)
    F = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
    W = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for f in range(2):
        d, c = seq.frame(f)
        dd = torch.from_numpy(d.view(np.int16)).cuda()
        vol.integrate(dd, torch.from_numpy(c).cuda(), seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        T.tsdf_integrate_geometry_static(dims, s, mu, mw, _origin(dims, s), F, W, dd, seq.K_depth, seq.poses[f],
                                         stream)
        torch.cuda.synchronize()
        Fr, Wr, _ = vol.read()
        np.testing.assert_array_equal(W.cpu().numpy(), Wr, err_msg="weights after call %d" % (f + 1))
        assert float(np.abs(F.cpu().numpy() - Fr).max()) <= F_TOL
        assert (Wr > 0).sum() > 10000
    vol.close()


def test_static_entry_equals_the_oracle():
    """Four frames through the static entry against the oracle's geometry
    update (Section III): weights bit for bit, TSDF within 1e-5 (exact)."""
    dims = (88, 72, 64)
    seq = synth.sequence_small(n_frames=4, dims_geo=dims[0], seed=23)
    s = float(np.float32(1.0 / dims[0]))
    mu = float(np.float32(3 * s))
    mw = seq.max_weight
    origin = _origin(dims, s)
    o = oracle.Oracle(dims, dims, s, mu, mw, origin=origin)
    F = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
    W = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for f in range(4):
        d, _ = seq.frame(f)
        o.integrate_geometry(d, seq.K_depth, seq.poses[f])
        T.tsdf_integrate_geometry_static(dims, s, mu, mw, origin, F, W, torch.from_numpy(d.view(np.int16)).cuda(),
                                         seq.K_depth, seq.poses[f], stream)
    torch.cuda.synchronize()
    Fg, Wg = F.cpu().numpy(), W.cpu().numpy()
    np.testing.assert_array_equal(Wg, o.W)
    assert float(np.abs(Fg - o.F).max()) <= F_TOL
    assert np.array_equal(Fg, o.F)
    assert (Wg > 0).sum() > 10000


def test_static_entry_allocates_no_device_memory():
    """After a first call (which looks up the scratch array's address), more
    calls change neither the driver's free device memory nor the number of
    allocations PyTorch's caching allocator has made."""
    dims = (96, 80, 72)
    seq = synth.sequence_small(n_frames=3, dims_geo=dims[0], seed=22)
    s = float(np.float32(1.0 / dims[0]))
    F = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
    W = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.uint8, device="cuda")
    frames = [torch.from_numpy(seq.frame(f)[0].view(np.int16)).cuda() for f in range(3)]
    stream = torch.cuda.current_stream().cuda_stream
    args = (dims, s, float(np.float32(3 * s)), seq.max_weight, _origin(dims, s), F, W)
    T.tsdf_integrate_geometry_static(*args, frames[0], seq.K_depth, seq.poses[0], stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n0 = torch.cuda.memory_stats()["allocation.all.allocated"]
    for f in (1, 2, 1):
        T.tsdf_integrate_geometry_static(*args, frames[f], seq.K_depth, seq.poses[f], stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == n0
    assert int((W > 0).sum()) > 10000


def test_static_entry_rejects_host_and_mistyped_arrays():
    """Host arrays are refused by the library itself (TSDF_ERR_INVALID_ARG,
    nothing queued) and by the binding, which also checks dtypes and sizes."""
    import ctypes

    dims = (32, 32, 32)
    n = 32 ** 3
    Fh = np.zeros(n, np.float32)
    Wh = np.zeros(n, np.uint8)
    Dd = torch.zeros((48, 64), dtype=torch.int16, device="cuda")
    Fd = torch.zeros(n, dtype=torch.float32, device="cuda")
    Wd = torch.zeros(n, dtype=torch.uint8, device="cuda")
    Kd = np.ascontiguousarray(synth.K_DEPTH, np.float32).reshape(9)
    Tw = np.ascontiguousarray(np.eye(4), np.float32).reshape(16)
    fp = ctypes.POINTER(ctypes.c_float)
    lib = T.load()
    dv = (ctypes.c_int32 * 3)(*dims)
    org = (ctypes.c_float * 3)(-0.16, -0.16, 0.2)
    for f_ptr, w_ptr in ((Fh.ctypes.data, Wd.data_ptr()), (Fd.data_ptr(), Wh.ctypes.data)):
        st = lib.tsdf_integrate_geometry_static(dv, ctypes.c_float(0.01), ctypes.c_float(0.03), 64, org,
                                                ctypes.c_void_p(f_ptr), ctypes.c_void_p(w_ptr),
                                                ctypes.c_void_p(Dd.data_ptr()), T.tsdf_image_size(64, 48),
                                                Kd.ctypes.data_as(fp), Tw.ctypes.data_as(fp), None)
        assert st == T.TSDF_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        T.tsdf_integrate_geometry_static(dims, 0.01, 0.03, 64, (-0.16, -0.16, 0.2), Fd.cpu(), Wd, Dd, Kd, np.eye(4))
    with pytest.raises(ValueError):
        T.tsdf_integrate_geometry_static(dims, 0.01, 0.03, 64, (-0.16, -0.16, 0.2), Fd[:-1], Wd, Dd, Kd, np.eye(4))
    with pytest.raises(ValueError):
        T.tsdf_integrate_geometry_static(dims, 0.01, 0.03, 64, (-0.16, -0.16, 0.2), Fd, Wd.float(), Dd, Kd, np.eye(4))


def test_static_entry_rejects_sizes_beyond_its_scratch():
    import ctypes

    # 1024^3 voxels = 2,097,152 bricks > TSDF_STATIC_MAX_BRICKS; the arrays are
    # never touched (the size check comes first), so they are small here and
    # the raw C entry point is called
    lib = T.load()
    F = torch.zeros(1, dtype=torch.float32, device="cuda")
    W = torch.zeros(1, dtype=torch.uint8, device="cuda")
    d = torch.zeros((480, 640), dtype=torch.int16, device="cuda")
    Kd = np.ascontiguousarray(synth.K_DEPTH, np.float32).reshape(9)
    Tw = np.ascontiguousarray(np.eye(4), np.float32).reshape(16)
    fp = ctypes.POINTER(ctypes.c_float)

    def call(dims, depth):
        h, w = depth.shape
        return lib.tsdf_integrate_geometry_static((ctypes.c_int32 * 3)(*dims), ctypes.c_float(0.002),
                                                  ctypes.c_float(0.006), 64, (ctypes.c_float * 3)(-1, -1, -1),
                                                  ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                                  ctypes.c_void_p(depth.data_ptr()), T.tsdf_image_size(w, h),
                                                  Kd.ctypes.data_as(fp), Tw.ctypes.data_as(fp), None)

    assert call((1024, 1024, 1024), d) == T.TSDF_ERR_INVALID_ARG
    big = torch.zeros((4200, 4200), dtype=torch.int16, device="cuda")  # > TSDF_STATIC_MAX_DEPTH_TILES tiles
    assert call((64, 64, 64), big) == T.TSDF_ERR_INVALID_ARG
