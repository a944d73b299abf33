"""Parity at the benchmark sizes under the strict error rule (no arithmetic
floor): the whole batch runs on the GPU and the oracle evaluates, over the full
join, every aggregate of the snowflake and Chow-Liu/cube batches and a seeded
sample of the tree batch."""
import numpy as np
import pytest

from oracle import oracle
from workloads import config2, config3, config4

from lmf_testlib import compare, run_engine

pytestmark = pytest.mark.gpu


def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return sorted(set([0] + rng.choice(n, size=min(k, n), replace=False).tolist()))


_C2_CACHE = {}


def _config2_full(order):
    """The 20M-row snowflake and the oracle over all of its 851 aggregates."""
    if order not in _C2_CACHE:
        sch, batch = config2(20_000_000, fact_order=order)
        _C2_CACHE.clear()
        _C2_CACHE[order] = (sch, batch, oracle.evaluate(sch, batch))
    return _C2_CACHE[order]


@pytest.mark.parametrize('order,precision,key_level', [('sorted', 0, True), ('sorted', 0, False), ('sorted', 1, True),
                                                       ('random', 0, False), ('random', 1, True)])
def test_config2_full_size(order, precision, key_level):
    """Every aggregate of the benchmark batch, both fact orders, the key-level
    and the row-level FP32 Gram and the split-bf16 tensor-core Gram."""
    sch, batch, want = _config2_full(order)
    got, info, eng = run_engine(sch, batch, precision=precision, batching=1, key_level=key_level)
    assert info['precision'] == precision and info['root_rows'] == 20_000_000
    # the key-level form needs a foreign key in runs: the sorted order has them
    assert info['key_level'] == (1 if precision == 0 and key_level and order == 'sorted' else 0)
    fails, stats = compare(got, want)
    assert not fails, (fails[:3], stats)
    eng.close()


def _node_subschema(sch, node):
    """The schema with the fact table cut to the rows on which every predicate
    of `node` holds (joined values followed through the dense dimension keys).
    The oracle still applies the predicates itself, so a wrong cut can only
    make the check fail, never pass."""
    from workloads import Column, Relation, Schema
    from workloads.schemas import _joined_sample
    fact = sch.rel(sch.root)
    rows = np.arange(fact.nrows)
    mask = np.ones(fact.nrows, dtype=bool)
    for attr, op, t in node:
        v = _joined_sample(sch, attr, rows).astype(np.float64)
        mask &= (v <= t) if op == 'le' else (v > t)
    cut = Relation(fact.name, [Column(c.name, c.role, c.data[mask], c.cat_domain) for c in fact.columns])
    rels = [cut if r.name == sch.root else r for r in sch.relations]
    return Schema(rels, sch.edges, sch.root, dict(sch.meta)), int(mask.sum())


def test_config3_full_size():
    """10M rows, 64 nodes: four whole nodes (every feature x threshold x
    moment aggregate of each, ~1.9k per node), plus a seeded sample of 300
    aggregates from anywhere in the batch."""
    sch, batch = config3(10_000_000)
    got, info, eng = run_engine(sch, batch, precision=1, batching=1)
    eng.close()
    assert info['tree_nodes'] == 64 and info['tree_groups'] == 1
    nodes = sch.meta['nodes']
    per_node = len(batch) // len(nodes)
    assert per_node * len(nodes) == len(batch)
    rng = np.random.default_rng(5)
    for ni in sorted(rng.choice(len(nodes), size=4, replace=False).tolist()):
        sub, n_rows = _node_subschema(sch, nodes[ni])
        idx = list(range(ni * per_node, (ni + 1) * per_node))
        assert all(batch[i].factors[:len(nodes[ni])] == nodes[ni] for i in idx)
        want = oracle.evaluate(sub, [batch[i] for i in idx])
        fails, stats = compare([got[i] for i in idx], want)
        assert not fails, (ni, n_rows, fails[:3], stats)
        assert all(0 <= got[i][0] <= n_rows for i in idx[::3])      # COUNTs within the node
    idx = _sample(len(batch), 300, 11)
    want = oracle.evaluate(sch, [batch[i] for i in idx])
    fails, stats = compare([got[i] for i in idx], want)
    assert not fails, (fails[:3], stats)


def test_config4_full_size_exact():
    """50M-row Chow-Liu pair counts, marginals and the data cube: every count
    bit-exact."""
    sch, batch = config4(50_000_000)
    got, info, eng = run_engine(sch, batch, precision=0, batching=1)
    assert info['root_rows'] == 50_000_000
    fails, stats = compare(got, oracle.evaluate(sch, batch))
    assert not fails, fails[:3]
    eng.close()


@pytest.mark.parametrize('order', ['sorted', 'random'])
def test_config4_reduced_exact(order):
    """Chow-Liu pair counts, marginals and the data cube: bit-exact counts."""
    sch, batch = config4(400_000, fact_order=order)
    got, info, eng = run_engine(sch, batch, precision=1, batching=1)
    want = oracle.evaluate(sch, batch)
    fails, stats = compare(got, want)
    assert not fails, fails[:3]
    eng.close()


def test_many_per_row_tables_exact():
    """More per-row tables than ride in the kernel parameters (96): 3-way
    COUNT tables over categories of three different keys, read by the
    compiled and the interpreted scan from the device descriptor array."""
    import itertools
    from workloads import Agg
    sch, _ = config4(100_003)
    cats = sch.meta['cats']
    dim = {c: c.split('_')[0] for c in cats}
    dom = {c: sch.owner(c).col(c).cat_domain for c in cats}
    triples = [t for t in itertools.combinations(cats, 3)
               if len({dim[c] for c in t}) == 3 and dom[t[0]] * dom[t[1]] * dom[t[2]] <= 20_000]
    assert len(triples) >= 130
    batch = [Agg(group_by=t) for t in triples[:130]]
    want = oracle.evaluate(sch, batch)
    for jit in (True, False):
        got, info, eng = run_engine(sch, batch, precision=0, batching=1, jit=jit)
        assert info['jit'] == int(jit)
        fails, _ = compare(got, want)
        assert not fails, fails[:3]
        eng.close()
