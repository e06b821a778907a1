"""The allocation-free geometry entry point against the regular one.

tsdf_integrate_geometry_static is for callers that cannot allocate device
memory (another framework owns the allocator, or the device-memory budget is
fixed in advance): they pass their own TSDF and weight arrays and the library
uses a fixed scratch array compiled into it.  Its results must equal the
geometry volume that tsdf_integrate produces, call after call.
"""
import numpy as np
import pytest

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


def test_static_entry_rejects_sizes_beyond_its_scratch():
    dims = (1024, 1024, 1024)  # 2,097,152 bricks > TSDF_STATIC_MAX_BRICKS
    F = torch.zeros(1, dtype=torch.float32, device="cuda")
    W = torch.zeros(1, dtype=torch.uint8, device="cuda")
    d = torch.zeros((480, 640), dtype=torch.int16, device="cuda")
    K = synth.K_DEPTH
    with pytest.raises(T.TsdfError) as e:
        T.tsdf_integrate_geometry_static(dims, 0.002, 0.006, 64, (-1, -1, -1), F, W, d, K, np.eye(4), None)
    assert e.value.status == T.TSDF_ERR_INVALID_ARG
    big = torch.zeros((4200, 4200), dtype=torch.int16, device="cuda")  # > TSDF_STATIC_MAX_DEPTH_TILES tiles
    with pytest.raises(T.TsdfError) as e:
        T.tsdf_integrate_geometry_static((64, 64, 64), 0.01, 0.03, 64, (-0.3, -0.3, -0.3), F, W, big, K, np.eye(4),
                                         None)
    assert e.value.status == T.TSDF_ERR_INVALID_ARG
