"""Pins for the CPU oracle: checks against things other than the oracle itself.

* brute force: the natural join as the filtered cartesian product of all
  relations (every attribute name shared by two relations must agree), with
  each aggregate summed exactly (math.fsum / Python ints);
* a hand-worked example stored under tests/golden/ (Example 3.1's shape);
* special cases that reduce to library routines (one relation: X^T X by numpy);
* closed forms (COUNT = fact rows when every foreign key has exactly one
  match; dimension sums = sum_k x[k] * histogram(k));
* invariants of the definitions: Gram symmetric positive semi-definite, grouped
  results marginalise to the ungrouped ones, pair/cube tables marginalise,
  tree-node counts are monotone in the threshold and partition the join;
* the chain example of Sec. 3.3, whose per-value counts are products of the
  left and right views L_i * R_i;
* the aggregate-count formulas of Sec. 2.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle
from oracle_pinlib import (assert_close, brute_force, check_against_brute_force,
                           check_compensated_sum, shared_attribute_schema)
from workloads import (Agg, Column, Relation, Schema, chain_schema, config1, config2,
                       config3, config4, covar_batch, cube_batch, pair_count_batch,
                       spread_keys, tiny_schema)

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


# ----------------------------------------------------------------------------
@pytest.mark.parametrize('seed', list(range(40)))
def test_brute_force_tiny(seed):
    sch, batch = tiny_schema(1000 + seed, unique_keys=(seed % 4 == 3))
    check_against_brute_force(sch, batch, nthreads=1 + seed % 3)


@pytest.mark.parametrize('seed', list(range(12)))
def test_brute_force_tiny_float32(seed):
    """FP32 feature columns (the benchmark's dtype) are read exactly."""
    sch, batch = tiny_schema(1000 + seed, feat_dtype=np.float32)
    check_against_brute_force(sch, batch, nthreads=1 + seed % 2)


@pytest.mark.parametrize('seed', list(range(3)))
def test_join_on_two_shared_attributes(seed):
    """A child sharing two attributes with its parent joins on both."""
    sch, batch = shared_attribute_schema(seed)
    check_against_brute_force(sch, batch, nthreads=1 + seed % 2)
    # the pin has teeth: joined on the key alone, the join is larger
    S = sch.rel('S')
    renamed = Relation('S', [Column('b2' if c.name == 'b' else c.name, c.role, c.data,
                                    c.cat_domain) for c in S.columns])
    key_only = Schema([sch.rel('R'), renamed, sch.rel('U')], sch.edges, sch.root)
    _, size, _ = brute_force(sch, [Agg()])
    _, size_key_only, _ = brute_force(key_only, [Agg()])
    assert size_key_only > size > 0


@pytest.mark.parametrize('seed', list(range(8)))
def test_sparse_keys_same_results(seed):
    """An injective relabelling of the join keys (values ~1e6 apart) changes
    no aggregate: the join depends on key equality only (Sec. 1.1)."""
    sch, batch = tiny_schema(1000 + seed)
    sp = spread_keys(sch)
    assert all(c.data.max() > 1_000_000 for r in sp.relations for c in r.columns
               if c.role == 'key' and r.nrows and c.data.max() > 0)
    check_against_brute_force(sp, batch, nthreads=1 + seed % 3)
    a, b = oracle.evaluate(sch, batch), oracle.evaluate(sp, batch)
    assert a.join_size == b.join_size
    for x, y in zip(a.values, b.values):
        assert np.array_equal(x, y)


@pytest.mark.parametrize('nthreads', [1, 3])
def test_compensated_sum_is_exact(nthreads):
    """Terms of size 1e16 that cancel down to 4: the compensated sum is exact."""
    check_compensated_sum(nthreads=nthreads)


def test_brute_force_covers_fanout_and_dangling():
    """The tiny generator must actually produce duplicate keys, dangling keys,
    empty relations and joins larger than the root (otherwise the brute-force
    pin would not exercise them)."""
    seen = {'fanout': False, 'dangling': False, 'empty': False}
    for seed in range(40):
        sch, batch = tiny_schema(1000 + seed, unique_keys=(seed % 4 == 3))
        root_rows = sch.rel(sch.root).nrows
        _, size, _ = brute_force(sch, [Agg()])
        seen['fanout'] |= size > root_rows
        seen['dangling'] |= size < root_rows
        seen['empty'] |= any(r.nrows == 0 for r in sch.relations)
    assert all(seen.values()), seen


def test_threads_deterministic():
    sch, batch = config1(5000)
    a = oracle.evaluate(sch, batch, nthreads=3)
    b = oracle.evaluate(sch, batch, nthreads=3)
    for x, y in zip(a.values, b.values):
        assert np.array_equal(x, y)


# ----------------------------------------------------------------------------
def _load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    rels = []
    for rname, cols in g['relations'].items():
        cs = []
        for cname, spec in cols.items():
            dt = np.int32 if spec['role'] in ('key', 'cat') else np.float64
            cs.append(Column(cname, spec['role'], np.array(spec['values'], dt),
                             spec.get('domain', 0)))
        rels.append(Relation(rname, cs))
    sch = Schema(rels, [tuple(e) for e in g['edges']], g['root'])
    batch = [Agg(tuple(q['group_by']), tuple(tuple(f) for f in q['factors']))
             for q in g['queries']]
    return sch, batch, g['expected']


def test_golden_hand_worked_example():
    sch, batch, expected = _load_golden('favorita_toy.json')
    res = oracle.evaluate(sch, batch, nthreads=1)
    for a, want in enumerate(expected):
        got = res.values[a]
        if res.kinds[a] == 'count':
            assert got.tolist() == want, (a, got, want)
        else:
            assert_close(got, np.array(want, np.float64))


# ----------------------------------------------------------------------------
def test_single_relation_gram_matches_numpy():
    """One relation, no join: the covar batch is X^T X with a constant column."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((3000, 5))
    rel = Relation('R', [Column(f'x{i}', 'cont', X[:, i].copy()) for i in range(5)])
    sch = Schema([rel], [], 'R')
    feats = [f'x{i}' for i in range(5)]
    batch = covar_batch(feats)
    res = oracle.evaluate(sch, batch)
    Z = np.hstack([np.ones((3000, 1)), X])
    G = Z.T @ Z
    k = 0
    assert res.values[0][0] == 3000
    k = 1
    for i in range(5):
        assert_close(res.values[k], [G[0, i + 1]], rel=1e-11)
        k += 1
    for i in range(5):
        for j in range(i, 5):
            assert_close(res.values[k], [G[i + 1, j + 1]], rel=1e-11)
            k += 1
    for i in range(5):
        assert abs(res.values[1 + i][0] - math.fsum(X[:, i])) <= 1e-12 * np.abs(X[:, i]).sum()


def test_count_is_fact_rows_and_dimension_marginals():
    """Every foreign key has exactly one dimension row, so |join| = N; a
    dimension feature's sum is sum_k x[k] * histogram of the foreign key."""
    sch, batch = config1(20000)
    res = oracle.evaluate(sch, batch)
    assert res.values[0][0] == 20000 and res.join_size == 20000
    R, S, T = sch.rel('R'), sch.rel('S'), sch.rel('T')
    h1 = np.bincount(R.col('k1').data, minlength=1000)
    h2 = np.bincount(R.col('k2').data, minlength=500)
    feats = sch.meta['features']
    for name, rel, h in [('s0', S, h1), ('s3', S, h1), ('t0', T, h2), ('t2', T, h2)]:
        a = batch.index(Agg(factors=((name, 'pow', 1),)))
        want = math.fsum(rel.col(name).data * h)
        assert abs(res.values[a][0] - want) <= 1e-12 * res.abs[a][0]
        a2 = batch.index(Agg(factors=((name, 'pow', 2),)))
        want2 = math.fsum(rel.col(name).data ** 2 * h)
        assert abs(res.values[a2][0] - want2) <= 1e-12 * res.abs[a2][0]
    # a cross term between two dimensions through the co-occurrence of keys
    co = np.zeros((1000, 500))
    np.add.at(co, (R.col('k1').data, R.col('k2').data), 1.0)
    a = batch.index(Agg(factors=(('s1', 'pow', 1), ('t1', 'pow', 1))))
    want = float(S.col('s1').data @ co @ T.col('t1').data)
    assert abs(res.values[a][0] - want) <= 1e-11 * res.abs[a][0]
    assert len(feats) == 10


def _gram(res, batch, feats):
    n = len(feats)
    G = np.zeros((n + 1, n + 1))
    idx = {f: i + 1 for i, f in enumerate(feats)}
    for a, agg in enumerate(batch):
        if agg.group_by:
            continue
        if not agg.factors:
            G[0, 0] = res.values[a][0]
        elif len(agg.factors) == 1 and agg.factors[0][2] == 1:
            i = idx[agg.factors[0][0]]
            G[0, i] = G[i, 0] = res.values[a][0]
        elif len(agg.factors) == 1:
            i = idx[agg.factors[0][0]]
            G[i, i] = res.values[a][0]
        else:
            i, j = idx[agg.factors[0][0]], idx[agg.factors[1][0]]
            G[i, j] = G[j, i] = res.values[a][0]
    return G


def test_gram_is_psd():
    sch, batch = config1(20000)
    res = oracle.evaluate(sch, batch)
    G = _gram(res, batch, sch.meta['features'])
    np.linalg.cholesky(G)              # raises unless positive definite
    assert np.all(np.linalg.eigvalsh(G) > 0)


# ----------------------------------------------------------------------------
def test_grouped_and_pairs_marginalise():
    sch, batch = config2(30000)
    res = oracle.evaluate(sch, batch)
    ung = {a.factors: res.values[i] for i, a in enumerate(batch) if not a.group_by}
    singles = {}
    for i, agg in enumerate(batch):
        if len(agg.group_by) == 1:
            tot = res.values[i].sum()
            want = ung[agg.factors][0]
            if res.kinds[i] == 'count':
                assert tot == want
                singles[agg.group_by[0]] = res.values[i]
            else:
                assert abs(math.fsum(res.values[i]) - want) <= 1e-12 * res.abs[i].sum()
    for i, agg in enumerate(batch):
        if len(agg.group_by) == 2:
            t = res.values[i].reshape(res.shapes[i])
            assert np.array_equal(t.sum(axis=1), singles[agg.group_by[0]])
            assert np.array_equal(t.sum(axis=0), singles[agg.group_by[1]])
    assert res.values[0][0] == 30000


def test_cube_marginalises():
    sch, _ = config4(40000)
    cube = sch.meta['cube']
    batch = cube_batch(cube)
    res = oracle.evaluate(sch, batch)
    full = res.values[-1].reshape(res.shapes[-1])
    for i, agg in enumerate(batch):
        axes = tuple(k for k, c in enumerate(cube) if c not in agg.group_by)
        want = full.sum(axis=axes) if axes else full
        assert np.array_equal(res.values[i].reshape(np.shape(want)), want)
    assert res.values[0][0] == 40000


def test_tree_level_invariants():
    sch, batch = config3(20000, sample_rows=20000)
    nodes = sch.meta['nodes']
    feats = sch.meta['features']
    nt = len(sch.meta['thresholds'][feats[0]])
    # a small sample of (node, feature) blocks plus the node totals
    pick_nodes = [0, 5, 33, 63]
    sub = []
    for nu in pick_nodes:
        sub.append(Agg(factors=nodes[nu]))
        for f in feats[:3]:
            for t in sch.meta['thresholds'][f]:
                sub.append(Agg(factors=nodes[nu] + ((f, 'le', float(t)),)))
    res = oracle.evaluate(sch, sub)
    k = 0
    for nu in pick_nodes:
        total = res.values[k][0]
        k += 1
        for f in feats[:3]:
            m = len(sch.meta['thresholds'][f])
            c = np.array([res.values[k + j][0] for j in range(m)])
            k += m
            assert np.all(np.diff(c) >= 0) and c[-1] <= total
    # the 64 leaves partition the join
    tot = oracle.evaluate(sch, [Agg(factors=n) for n in nodes])
    assert sum(int(v[0]) for v in tot.values) == 20000
    assert nt <= 32


# ----------------------------------------------------------------------------
def test_chain_example_left_right_views():
    """Sec. 3.3: with root S_i for Q_i(X_i; 1), the count of each X_i value is
    L_i(X_i) * R_i(X_i), L from the right end of the chain and R from the left."""
    n, size, dom = 5, 12, 4
    sch = chain_schema(n, size, dom, seed=11)
    S = [None] + [sch.rel(f'S{k}') for k in range(1, n)]
    A = {k: S[k].columns[0].data for k in range(1, n)}   # X_k of S_k
    B = {k: S[k].columns[1].data for k in range(1, n)}   # X_{k+1} of S_k
    L = {n: np.ones(dom)}
    for i in range(n - 1, 0, -1):                        # L_i += S_i, L_{i+1}
        L[i] = np.zeros(dom)
        np.add.at(L[i], A[i], L[i + 1][B[i]])
    R = {1: np.ones(dom)}
    for i in range(2, n + 1):                            # R_i += S_{i-1}, R_{i-1}
        R[i] = np.zeros(dom)
        np.add.at(R[i], B[i - 1], R[i - 1][A[i - 1]])
    batch = [Agg(group_by=(f'X{i}',)) for i in range(1, n + 1)]
    res = oracle.evaluate(sch, batch)
    for i in range(1, n + 1):
        assert np.array_equal(res.values[i - 1], (L[i] * R[i]).astype(np.int64)), i
    want, size_bf, _ = brute_force(sch, batch)
    assert res.join_size == size_bf
    for i in range(n):
        assert np.array_equal(res.values[i], want[i])
    # the categorical copies G_i of the join attributes (the per-query-root
    # GPU tests group by them) give the same L_i * R_i counts
    sch_g = chain_schema(n, size, dom, seed=11, group_copies=True)
    batch_g = [Agg(group_by=(f'G{i}',)) for i in range(2, n)]
    res_g = oracle.evaluate(sch_g, batch_g)
    for i in range(2, n):
        assert np.array_equal(res_g.values[i - 2], (L[i] * R[i]).astype(np.int64)), i


# ----------------------------------------------------------------------------
def test_batch_size_formulas():
    """Sec. 2: (n+1)(n+2)/2 for the covar matrix; n(n-1)/2 pair counts for
    Chow-Liu; 2^d nu for a d-dimensional cube; d n (p+1) c for tree nodes."""
    _, b1 = config1(10)
    assert len(b1) == (10 + 1) * (10 + 2) // 2 == 66
    _, b2 = config2(10)
    assert len(b2) == 31 * 32 // 2 + 10 * 31 + 45 == 851
    sch3, b3 = config3(2000, sample_rows=2000)
    nthr = sum(len(v) for v in sch3.meta['thresholds'].values())
    assert len(b3) == 64 * nthr * 3
    _, b4 = config4(10)
    assert len(b4) == 30 * 29 // 2 + 30 + 2 ** 3 == 473
    assert len(pair_count_batch([str(i) for i in range(9)])) == 36


def _marginal_ok(res, batch, sch):
    R, S = sch.rel('R'), sch.rel('S')
    h1 = np.bincount(R.col('k1').data, minlength=1000)
    a = batch.index(Agg(factors=(('s0', 'pow', 1),)))
    return abs(res.values[a][0] - math.fsum(S.col('s0').data * h1)) <= 1e-12 * res.abs[a][0]


def _cross_ok(res, batch, sch):
    R, S, T = sch.rel('R'), sch.rel('S'), sch.rel('T')
    co = np.zeros((1000, 500))
    np.add.at(co, (R.col('k1').data, R.col('k2').data), 1.0)
    a = batch.index(Agg(factors=(('s1', 'pow', 1), ('t1', 'pow', 1))))
    return abs(res.values[a][0] - float(S.col('s1').data @ co @ T.col('t1').data)) \
        <= 1e-11 * res.abs[a][0]


def _pairs_ok(res, batch):
    singles = {a.group_by[0]: res.values[i] for i, a in enumerate(batch)
               if len(a.group_by) == 1 and not a.factors}
    for i, a in enumerate(batch):
        if len(a.group_by) == 2:
            t = res.values[i].reshape(res.shapes[i])
            if not (np.array_equal(t.sum(axis=1), singles[a.group_by[0]]) and
                    np.array_equal(t.sum(axis=0), singles[a.group_by[1]])):
                return False
    return True


def test_mutations_are_caught():
    """Plausible slips (a flipped sign, a dropped cross term, a transposed pair
    table, a group shifted by one) each break a pin above."""
    sch, batch = config1(3000)
    res = oracle.evaluate(sch, batch)
    assert _marginal_ok(res, batch, sch) and _cross_ok(res, batch, sch)
    a = batch.index(Agg(factors=(('s0', 'pow', 1),)))
    res.values[a] = -res.values[a]
    assert not _marginal_ok(res, batch, sch)
    c = batch.index(Agg(factors=(('s1', 'pow', 1), ('t1', 'pow', 1))))
    res.values[c] = res.values[c] * 0.0
    assert not _cross_ok(res, batch, sch)

    sch2, batch2 = config2(4000)
    res2 = oracle.evaluate(sch2, batch2)
    assert _pairs_ok(res2, batch2)
    for i, g in enumerate(batch2):
        if len(g.group_by) == 2 and res2.shapes[i][0] != res2.shapes[i][1]:
            saved = res2.values[i]
            res2.values[i] = saved.reshape(res2.shapes[i]).T.copy().reshape(-1)
            res2.shapes[i] = res2.shapes[i][::-1]
            assert not _pairs_ok(res2, batch2)
            res2.values[i] = saved
            res2.shapes[i] = res2.shapes[i][::-1]
            res2.values[i] = np.roll(saved, 1)
            assert not _pairs_ok(res2, batch2)
            break
