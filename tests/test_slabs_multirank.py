"""One scan split into z-slabs over ranks (the multi-GPU partition of one
volume), run as gloo ranks on the CPU with the oracle doing each rank's
integration: every rank holds its slab plus a one-voxel geometry margin,
receives every frame, and the slabs' own parts, gathered on rank 0 in z order,
must equal the whole-volume oracle bit for bit.  This checks the partition
(paper_1602_06645_gb300.slab_ranges, the held ranges) and that computing each
voxel at its global index makes the partition invisible in the results."""
import socket

import numpy as np
import pytest

import oracle
import paper_1602_06645_gb300 as T
from paper_1602_06645_gb300 import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _integrate(seq, n_frames, slab=None):
    o = oracle.Oracle(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, slab=slab)
    for f in range(n_frames):
        d, c = seq.frame(f)
        o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    return o


def _own_part(o, seq, slab):
    g0, _, _, _ = oracle.slab_extent(seq.dims_geo, seq.dims_col, *slab)
    a, b = slab[0] - g0, slab[1] - g0
    return o.F[a:b].copy(), o.W[a:b].copy(), o.C.copy()


def _rank_main(rank, world, port, dims, n_frames, out):
    import os

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seq = synth.sequence_small(n_frames=n_frames, dims_geo=dims)
        slab = T.slab_ranges(seq.dims_geo, seq.dims_col, world)[rank]
        part = _own_part(_integrate(seq, n_frames, slab), seq, slab)
        parts = [None] * world if rank == 0 else None
        dist.gather_object(part, parts, dst=0)
        if rank == 0:
            whole = _integrate(seq, n_frames)
            F = np.concatenate([p[0] for p in parts])
            W = np.concatenate([p[1] for p in parts])
            C = np.concatenate([p[2] for p in parts])
            out["equal"] = (np.array_equal(F.view(np.uint32), whole.F.view(np.uint32)) and
                            np.array_equal(W, whole.W) and np.array_equal(C, whole.C))
            out["observed"] = int((whole.W > 0).sum()), int(((whole.C >> 24) > 0).sum())
            # the cut runs through observed voxels of both volumes
            z = slab[1]
            out["cut_observed"] = int((whole.W[z - 1:z + 1] > 0).sum()), int(((whole.C[2 * z - 2:2 * z + 2] >> 24) > 0).sum())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_over_gloo_ranks_equal_the_whole_volume(world):
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), 48, 3, out), nprocs=world, join=True)
        res = dict(out)
    assert res["equal"]
    assert res["observed"][0] > 5000 and res["observed"][1] > 1000


def test_slab_ranges_cut_on_whole_colour_voxels_and_bricks():
    assert T.slab_ranges((64, 64, 64), (128, 128, 128), 2) == [(0, 32), (32, 64)]
    assert T.slab_ranges((512, 512, 512), (1024, 1024, 1024), 8) == [(64 * k, 64 * k + 64) for k in range(8)]
    r = T.slab_ranges((44, 44, 44), (88, 88, 88), 3)  # 44 layers: brick-aligned cuts where possible
    assert r[0][0] == 0 and r[-1][1] == 44 and all(a < b for a, b in r) and all(z % 8 == 0 for z, _ in r)
    # colour / geometry = 5 / 3: cuts on multiples of 3 geometry layers
    r = T.slab_ranges((30, 30, 30), (50, 50, 50), 2)
    assert all((z * 50) % 30 == 0 for s in r for z in s)
    with pytest.raises(ValueError):
        T.slab_ranges((8, 8, 8), (16, 16, 16), 9)


def test_slab_extent_margins():
    assert oracle.slab_extent((64, 64, 64), (128, 128, 128), 0, 32) == (0, 33, 0, 64)
    assert oracle.slab_extent((64, 64, 64), (128, 128, 128), 32, 64) == (31, 64, 64, 128)
    assert oracle.slab_extent((64, 64, 64), (128, 128, 128), 16, 40) == (15, 41, 32, 80)
    with pytest.raises(ValueError):
        oracle.slab_extent((30, 30, 30), (50, 50, 50), 10, 30)  # 10 * 50 / 30 is not whole
