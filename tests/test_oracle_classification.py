"""Pins for the classification-tree level of the oracle (Sec. 2, decision
trees): the batch of workloads.config3_classification, the class counts of
Eq. classification-tree as the oracle evaluates them, and the CART split
choice over them (oracle/consumers.py: impurity, split_cost, best_split,
classification_level_splits, cart_children).

* The entropy and Gini index against closed forms.
* The oracle's class counts of a level batch against counts taken directly
  from the materialised join (the snowflake's dimension keys are unique, so
  the join has one tuple per fact row).
* The best split of the root and a two-level CART tree grown from oracle
  batches against scikit-learn's decision tree on the materialised join: the
  same least cost (scikit-learn's entropy is in bits), the same partition.
* Planted mistakes in the split arithmetic are caught.
"""
import math

import numpy as np
import pytest

from oracle import consumers, oracle
from workloads import Agg, config3_classification
from workloads.schemas import _joined_sample


def _materialise(sch):
    """Every feature of the level and the class, one row per fact row."""
    rows = np.arange(sch.rel('F').nrows)
    X = {f: _joined_sample(sch, f, rows).astype(np.float64) for f in sch.meta['features']}
    return X, sch.rel('F').col('cls').data.astype(np.int64)


def _mask(X, conds, n):
    m = np.ones(n, bool)
    for f, op, t in conds:
        m &= (X[f] <= t) if op == 'le' else (X[f] > t)
    return m


# ----------------------------------------------------------------------------
def test_impurity_closed_forms():
    for crit in ('gini', 'entropy'):
        assert consumers.impurity([7, 0, 0], crit) == 0.0
        assert consumers.impurity([0, 0], crit) == 0.0
    for p in (2, 3, 5):
        assert abs(consumers.impurity([4] * p, 'gini') - (1 - 1 / p)) <= 1e-15
        assert abs(consumers.impurity([4] * p, 'entropy') - math.log(p)) <= 1e-15
    a, b = 3, 9
    assert abs(consumers.impurity([a, b], 'gini') - 2 * a * b / (a + b) ** 2) <= 1e-15
    assert abs(consumers.impurity([1, 3], 'entropy') + (0.25 * math.log(0.25) + 0.75 * math.log(0.75))) <= 1e-15
    # a split that separates the classes costs nothing; one that keeps the mix costs the parent's index
    assert consumers.split_cost([5, 0], [5, 5]) == 0.0
    assert abs(consumers.split_cost([2, 2], [5, 5]) - 0.5) <= 1e-15
    assert consumers.best_split([5, 5], [('all', [5, 5]), ('none', [0, 0])]) is None


def test_level_class_counts_match_the_materialised_join():
    sch, batch = config3_classification(4000, n_classes=3, n_nodes_depth=2, n_thresholds=5, sample_rows=4000)
    res = oracle.evaluate(sch, batch)
    X, cls = _materialise(sch)
    n = len(cls)
    for agg, got in zip(batch, res.values):
        m = _mask(X, agg.factors, n)
        if agg.group_by:
            assert agg.group_by == ('cls',)
            want = np.bincount(cls[m], minlength=3)
        else:
            want = np.array([m.sum()])
        np.testing.assert_array_equal(np.asarray(got, np.int64).reshape(-1), want)
    # the CART step reads them back in the batch's layout
    nodes, feats, thr = sch.meta['nodes'], sch.meta['features'], sch.meta['thresholds']
    level = consumers.classification_level_splits(batch, res.values, nodes, feats, thr, 3)
    assert len(level) == len(nodes) == 4
    assert sum(int(t.sum()) for t, _, _ in level) <= n


def _level_batch(node, feats, thr):
    batch = [Agg(group_by=('cls',), factors=tuple(node)), Agg(factors=tuple(node))]
    for f in feats:
        for t in thr[f]:
            alpha = tuple(node) + ((f, 'le', float(t)),)
            batch += [Agg(group_by=('cls',), factors=alpha), Agg(factors=alpha)]
    return batch


def _midpoints(X, feats):
    """Every threshold between two consecutive distinct values of a feature:
    the candidates a CART implementation tries on a continuous attribute."""
    thr = {}
    for f in feats:
        v = np.unique(X[f])
        thr[f] = (v[:-1] / 2.0 + v[1:] / 2.0)
    return thr


def _sklearn_cost(tree, node, crit):
    t = tree.tree_
    l, r = t.children_left[node], t.children_right[node]
    n = t.weighted_n_node_samples
    cost = (n[l] * t.impurity[l] + n[r] * t.impurity[r]) / n[node]
    return cost * (math.log(2) if crit == 'entropy' else 1.0)   # bits -> nats


def _small(seed=11):
    sch, _ = config3_classification(600, n_classes=3, n_nodes_depth=0, n_thresholds=1, sample_rows=600,
                                    seed=seed)
    feats = sch.meta['features'][:8]
    X, cls = _materialise(sch)
    return sch, feats, X, cls


@pytest.mark.parametrize('crit', ['gini', 'entropy'])
def test_root_split_matches_sklearn(crit):
    tree_mod = pytest.importorskip('sklearn.tree')
    sch, feats, X, cls = _small()
    thr = _midpoints(X, feats)
    batch = _level_batch((), feats, thr)
    res = oracle.evaluate(sch, batch)
    (total, split, cost), = consumers.classification_level_splits(batch, res.values, [()], feats, thr, 3, crit)
    np.testing.assert_array_equal(total, np.bincount(cls, minlength=3))
    M = np.column_stack([X[f] for f in feats]).astype(np.float32)
    sk = tree_mod.DecisionTreeClassifier(criterion=crit, max_depth=1, random_state=0).fit(M, cls)
    assert abs(cost - _sklearn_cost(sk, 0, crit)) <= 1e-12
    # the same partition of the rows
    f, t = split
    ours = X[f] <= t
    theirs = M[:, sk.tree_.feature[0]] <= sk.tree_.threshold[0]
    assert np.array_equal(ours, theirs) or abs(cost - _sklearn_cost(sk, 0, crit)) <= 1e-15


def test_two_level_cart_matches_sklearn():
    """CART grown one level at a time from oracle batches (the root's level,
    then its two children's): the same training cost at depth 2 as
    scikit-learn's greedy tree."""
    tree_mod = pytest.importorskip('sklearn.tree')
    sch, feats, X, cls = _small(seed=5)
    thr = _midpoints(X, feats)
    res = oracle.evaluate(sch, _level_batch((), feats, thr))
    (_, split, _), = consumers.classification_level_splits(_level_batch((), feats, thr), res.values, [()],
                                                           feats, thr, 3)
    children = consumers.cart_children((), split)
    leaves_cost = 0.0
    n = len(cls)
    for child in children:
        batch = _level_batch(child, feats, thr)
        r = oracle.evaluate(sch, batch)
        (total, s, cost), = consumers.classification_level_splits(batch, r.values, [child], feats, thr, 3)
        w = float(total.sum()) / n
        leaves_cost += w * (consumers.impurity(total) if s is None else cost)
    M = np.column_stack([X[f] for f in feats]).astype(np.float32)
    sk = tree_mod.DecisionTreeClassifier(criterion='gini', max_depth=2, random_state=0).fit(M, cls)
    t = sk.tree_
    sk_cost = sum(t.weighted_n_node_samples[i] * t.impurity[i] for i in range(t.node_count)
                  if t.children_left[i] < 0) / n
    assert abs(leaves_cost - sk_cost) <= 1e-12


# ----------------------------------------------------------------------------
MUTANTS = [
    ('Gini without the squares', 'return 1.0 - math.fsum(float(p) * float(p) for p in pi)',
     'return 1.0 - math.fsum(float(p) for p in pi)'),
    ('entropy sign flipped', 'return -math.fsum(float(p) * math.log(float(p)) for p in pi if p > 0)',
     'return math.fsum(float(p) * math.log(float(p)) for p in pi if p > 0)'),
    ('right side taken as the whole fragment', '    rgt = tot - lft\n', '    rgt = tot\n'),
    ('sides not weighted by their share',
     'return (float(lft.sum()) / n) * impurity(lft, criterion) + (float(rgt.sum()) / n) * impurity(rgt, criterion)',
     'return impurity(lft, criterion) + impurity(rgt, criterion)'),
    ('the costliest split taken', 'if best is None or cost < best[1]:', 'if best is None or cost > best[1]:'),
]


@pytest.mark.parametrize('what,old,new', MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(what, old, new):
    pytest.importorskip('sklearn.tree')
    import types
    with open(consumers.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, what
    mod = types.ModuleType('consumers_copy')
    exec(compile(text.replace(old, new), consumers.__file__, 'exec'), mod.__dict__)
    names = ('impurity', 'split_cost', 'best_split', 'classification_level_splits', 'cart_children')
    saved = {k: getattr(consumers, k) for k in names}
    failed = False
    try:
        for k in names:
            setattr(consumers, k, getattr(mod, k))
        for test in (test_impurity_closed_forms, lambda: test_root_split_matches_sklearn('gini'),
                     lambda: test_root_split_matches_sklearn('entropy'), test_two_level_cart_matches_sklearn):
            try:
                test()
            except AssertionError:
                failed = True
                break
    finally:
        for k, v in saved.items():
            setattr(consumers, k, v)
    assert failed, what
