"""Host-side logic of bench.py (no GPU): the quartet sampler used by the oracle
legs returns only significant canonical quartets, and the sampled class mix
follows the list."""
import numpy as np

import bench
import oracle
import workloads as W


def test_sampled_quartets_are_significant_and_canonical():
    basis, _ = W.workload(0)
    lists = bench._lists_without_gpu(basis)
    Q = lists["Q"]
    q = bench.sample_quartets(lists, basis, 500, seed=3)
    pidx = lambda a, b: a * (a + 1) // 2 + b
    for a, b, c, d in q:
        assert a >= b and c >= d
        assert float(Q[pidx(a, b)]) * float(Q[pidx(c, d)]) >= bench.THRESH
    o = oracle.Oracle(basis)
    assert o.quartet_batch(q[:20]) > 0.0
