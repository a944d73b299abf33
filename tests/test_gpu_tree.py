"""GPU parity of threshold-filtered aggregates (regression-tree node batches).

The whole batch of a tree level (64 nodes x 20 features x 32 thresholds x
{COUNT, SUM(y), SUM(y^2)}) is planned and run on the GPU; the oracle
re-evaluates a seeded sample of the aggregates literally (products of
indicators), and properties that hold for every aggregate are checked on the
full output (counts monotone in the threshold, node totals partition the join).
"""
import numpy as np
import pytest

from oracle import oracle
from workloads import Agg, config3, tiny_schema

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu


def _sample(batch, k, seed):
    rng = np.random.default_rng(seed)
    idx = sorted(set(rng.choice(len(batch), size=min(k, len(batch)), replace=False).tolist()))
    return idx


def test_tree_level_reduced_full_batch():
    sch, batch = config3(150_001, sample_rows=150_001)
    got, info, eng = run_engine(sch, batch, precision=1, batching=1)
    assert info['n_filtered_aggs'] == len(batch) == 64 * 20 * 32 * 3 or info['n_filtered_aggs'] == len(batch)
    idx = _sample(batch, 1500, 3)
    want = oracle.evaluate(sch, [batch[i] for i in idx])
    fails, stats = compare([got[i] for i in idx], want)
    assert not fails, (fails[:5], stats)
    # invariants over the full output: per (node, feature, moment) the values
    # over increasing thresholds are prefix sums (counts non-decreasing)
    nodes = sch.meta['nodes']
    feats = sch.meta['features']
    k = 0
    node_total = []
    for nu in range(len(nodes)):
        first_counts = []
        for f in feats:
            nt = len(sch.meta['thresholds'][f])
            cnt = np.array([got[k + 3 * j][0] for j in range(nt)])
            assert np.all(np.diff(cnt) >= 0)
            first_counts.append(cnt[-1])
            k += 3 * nt
        node_total.append(max(first_counts))
    assert sum(node_total) <= 150_001
    eng.close()


def test_tree_level_node_totals_partition():
    """Node conjunctions alone (one threshold factor dropped) sum to |join|."""
    sch, _ = config3(60_000, sample_rows=60_000)
    batch = [Agg(factors=n) for n in sch.meta['nodes']]
    got, info, eng = run_engine(sch, batch, precision=1, batching=0)
    assert sum(int(g[0]) for g in got) == 60_000
    want = oracle.evaluate(sch, batch)
    fails, _ = compare(got, want)
    assert not fails
    eng.close()


def test_tree_deterministic_and_graph():
    sch, batch = config3(80_000, sample_rows=80_000)
    batch = batch[: 3 * 32 * 20 * 4]      # four nodes
    outs, info, eng = run_engine(sch, batch, precision=1, batching=1, runs=3)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    want = oracle.evaluate(sch, batch)
    fails, stats = compare(outs[-1], want)
    assert not fails, (fails[:5], stats)
    eng.close()


@pytest.mark.parametrize('seed', list(range(12)))
def test_tiny_filtered(seed):
    """Filtered aggregates on tiny schemas, including fan-out and dangling keys;
    overlapping nodes (one predicate, or none left after the split) too."""
    sch, batch = tiny_schema(7000 + seed, unique_keys=(seed % 3 == 0), feat_dtype=np.float32)
    feats = sch.meta['features']
    f0 = feats[0]
    col = sch.owner(f0).col(f0).data
    if len(col) == 0:
        pytest.skip('empty relation holds the feature')
    ts = sorted(set(np.quantile(col, [0.25, 0.5, 0.75]).tolist()))
    aggs = []
    for t in ts:
        aggs.append(Agg(factors=((f0, 'le', t),)))
        aggs.append(Agg(factors=((f0, 'gt', t), (feats[-1], 'pow', 1))))
        aggs.append(Agg(factors=((f0, 'le', t), (feats[-1], 'le', ts[0]), (feats[0], 'pow', 2))))
    from paper_1906_08687_gb300 import LmfError
    # attributes below a fanning-out key cannot be thresholded per root row
    fanout_above = False
    for attr in {f0, feats[-1]}:
        rel = sch.owner(attr).name
        while rel != sch.root:
            parent, key = next((p, k) for p, c, k in sch.edges if c == rel)
            keys = sch.rel(rel).col(key).data
            fanout_above |= len(keys) > 0 and np.bincount(keys).max() > 1
            rel = parent
    if fanout_above:
        with pytest.raises(LmfError) as e:
            run_engine(sch, aggs, precision=0, batching=0)
        assert e.value.status == -10
        return
    got, info, eng = run_engine(sch, aggs, precision=0, batching=0)
    want = oracle.evaluate(sch, aggs)
    fails, stats = compare(got, want, arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:5], stats)
    eng.close()
