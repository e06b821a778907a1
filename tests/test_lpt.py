"""Longest-processing-time-first split of independent scans over devices
(paper_1602_06645_gb300.lpt_assign): host logic, checked on the CPU against
Graham's bound for the greedy rule, its tight worst case and brute force."""
import itertools
import random

import pytest

import paper_1602_06645_gb300 as T


def makespan(costs, parts):
    return max(sum(costs[i] for i in p) for p in parts)


def optimum(costs, n):
    """Smallest makespan over every assignment (brute force, tiny inputs)."""
    best = float("inf")
    for a in itertools.product(range(n), repeat=len(costs)):
        load = [0.0] * n
        for i, d in enumerate(a):
            load[d] += costs[i]
        best = min(best, max(load))
    return best


def test_graham_tight_case():
    # two devices, jobs 3 3 2 2 2: the greedy rule gives 7 against the optimum 6
    # (3 + 3 | 2 + 2 + 2), exactly (4/3 - 1/6) * 6
    costs = [3, 3, 2, 2, 2]
    parts = T.lpt_assign(costs, 2)
    assert parts == [[0, 2, 4], [1, 3]]
    assert makespan(costs, parts) == 7 and optimum(costs, 2) == 6


@pytest.mark.parametrize("seed", range(12))
def test_partition_and_bound_against_brute_force(seed):
    rng = random.Random(seed)
    n = rng.choice([2, 3])
    costs = [rng.randint(1, 40) for _ in range(rng.randint(n, 8))]
    parts = T.lpt_assign(costs, n)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    assert all(p == sorted(p) for p in parts)
    opt = optimum(costs, n)
    assert makespan(costs, parts) <= (4.0 / 3.0 - 1.0 / (3 * n)) * opt + 1e-9


def test_batched_scans_split():
    from paper_1602_06645_gb300 import synth
    edges = synth.batched_edges(64)
    costs = [9 * e ** 3 for e in edges]
    for n in (1, 2, 4, 8):
        parts = T.lpt_assign(costs, n)
        assert len(parts) == n and sorted(i for p in parts for i in p) == list(range(64))
        # no device is more than the largest scan above an even share
        assert makespan(costs, parts) <= sum(costs) / n + max(costs)
    assert T.lpt_assign(costs, 1) == [list(range(64))]
    assert T.lpt_assign([], 3) == [[], [], []]


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        T.lpt_assign([1, 2], 0)
    with pytest.raises(ValueError):
        T.lpt_assign([1, -2], 2)
    with pytest.raises(ValueError):
        T.lpt_assign([1, float("nan")], 2)
