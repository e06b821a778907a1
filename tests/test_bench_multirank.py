"""Host logic of bench.py for N > 1 ranks, run as two gloo ranks on the CPU.

With N ranks each GPU integrates its own scan (a different seed per rank, no
exchange on the data path); the job's time is the slowest rank's and its
units are the sum over ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        units = 1000.0 * (rank + 1)
        (mx,), (sm,) = bench.reduce_over_ranks(dist, "cpu", [ms], [units])
        (e2e,), _ = bench.reduce_over_ranks(dist, "cpu", [0.5 + rank])
        seq = bench.make_sequence("small", 2, rank)
        d, _ = seq.frame(0)
        out[rank] = (mx, sm, e2e, seq.seed, int(d.sum()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, sm, e2e, _, _ = res[r]
        assert mx == 15.0 and sm == 3000.0 and e2e == 1.5
    # each rank integrates its own scan: different seeds, different frames
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", [3.0], [7.0]) == ([3.0], [7.0])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(workload="small", steps=1, warmup=0, gpus=2))()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def _rank_batched(rank, world, port, out):
    import bench
    import paper_1602_06645_gb300 as T
    from paper_1602_06645_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        edges = synth.batched_edges(64)
        mine = T.lpt_assign([9 * e ** 3 for e in edges], world)[rank]
        units = sum(9 * edges[i] ** 3 for i in mine)
        (mx,), (total, count) = bench.reduce_over_ranks(dist, "cpu", [float(units)], [float(units), len(mine)])
        out[rank] = (tuple(mine), mx, total, count)
    finally:
        dist.destroy_process_group()


def test_batched_scans_split_over_two_gloo_ranks():
    """bench.py --workload batched with N ranks: each rank takes its longest-
    processing-time-first share of the 64 scans (computed locally, no
    exchange); the shares are disjoint and cover every scan, and the job's
    units are their sum."""
    from paper_1602_06645_gb300 import synth
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_batched, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    edges = synth.batched_edges(64)
    shares = [set(res[r][0]) for r in range(world)]
    assert not (shares[0] & shares[1]) and (shares[0] | shares[1]) == set(range(64))
    total = sum(9 * e ** 3 for e in edges)
    for r in range(world):
        assert res[r][2] == total and res[r][3] == 64
        assert res[r][1] <= total / world + 9 * max(edges) ** 3
