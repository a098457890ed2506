"""Cost-balanced split of a batch over devices (mlpf_shard_events, host only):
every event in exactly one shard, the LPT assignment reproduced by a brute-force
restatement of the rule, the makespan within 4/3 of the optimum found by
exhaustive search on small batches, and argument checks."""
import itertools

import numpy as np
import pytest

from paper_2601_17554_b300 import MlpfError, shard_events


def lpt_reference(sizes, k):
    cost = [int(n) ** 2 for n in sizes]
    order = sorted(range(len(sizes)), key=lambda e: (-cost[e], e))
    load, shard = [0] * k, [0] * len(sizes)
    for e in order:
        b = min(range(k), key=lambda j: (load[j], j))
        shard[e] = b
        load[b] += cost[e]
    return shard, load


@pytest.mark.parametrize("k", [1, 2, 3, 8])
def test_lpt_rule_and_costs(k):
    rng = np.random.default_rng(k)
    sizes = rng.integers(0, 5000, 57)
    shard, cost = shard_events(sizes, k)
    ref_shard, ref_load = lpt_reference(sizes, k)
    assert shard.tolist() == ref_shard
    assert cost.tolist() == [float(v) for v in ref_load]
    assert ((shard >= 0) & (shard < k)).all()
    np.testing.assert_allclose(cost.sum(), float((sizes.astype(np.float64) ** 2).sum()))


def test_lpt_within_four_thirds_of_optimum():
    rng = np.random.default_rng(7)
    for _ in range(20):
        sizes = rng.integers(1, 100, 9)
        _, cost = shard_events(sizes, 2)
        c = sizes.astype(np.int64) ** 2
        best = min(max(c[list(s)].sum(), c.sum() - c[list(s)].sum())
                   for r in range(len(c) + 1) for s in itertools.combinations(range(len(c)), r))
        assert cost.max() <= 4 / 3 * best + 1e-9


def test_more_shards_than_events_and_argument_checks():
    shard, cost = shard_events([10, 20], 4)
    assert sorted(shard.tolist()) == [0, 1] and cost.tolist() == [400.0, 100.0, 0.0, 0.0]
    shard, cost = shard_events([], 3)
    assert len(shard) == 0 and cost.tolist() == [0.0, 0.0, 0.0]
    with pytest.raises(MlpfError):
        shard_events([1, 2], 0)
    with pytest.raises(MlpfError):
        shard_events([1, -2], 2)
