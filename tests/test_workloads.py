"""The synthetic inputs follow their stated recipe: sizes, key ranges, value
distributions, input order and batch sizes of the seeded stand-ins for the
paper's datasets (Sec. 4, App. A), at reduced row counts."""
import numpy as np
import pytest

from workloads import (config1, config2, config3, config3_classification, config4, config5_schema,
                       many_to_many, sort_by_join_attributes, zipf_keys)
from workloads.schemas import Column, Relation, _rng


def _rank_slope(keys, k, top=100):
    """Slope of log frequency against log rank over the `top` most frequent keys."""
    cnt = np.sort(np.bincount(keys, minlength=k))[::-1][:top].astype(np.float64)
    r = np.arange(1, top + 1, dtype=np.float64)
    return np.polyfit(np.log(r), np.log(cnt), 1)[0]


@pytest.mark.parametrize('s', [0.8, 1.0, 1.1])
def test_zipf_keys_rank_frequency(s):
    keys = zipf_keys(_rng(5), 2_000_000, 1000, s)
    assert keys.dtype == np.int32 and keys.min() >= 0 and keys.max() < 1000
    assert abs(_rank_slope(keys, 1000) + s) < 0.06


def test_zipf_keys_uniform_and_permuted():
    keys = zipf_keys(_rng(6), 1_000_000, 500, 0.0)
    cnt = np.bincount(keys, minlength=500)
    expect = 1_000_000 / 500
    assert np.all(np.abs(cnt - expect) < 6 * np.sqrt(expect))
    # ranks go to key ids through a permutation: the hottest key is not id 0 in general
    hot = [int(np.argmax(np.bincount(zipf_keys(_rng(seed), 20000, 1000, 1.0), minlength=1000)))
           for seed in range(8)]
    assert len(set(hot)) > 1


def test_sort_by_join_attributes_order_and_rows():
    rng = _rng(9)
    n = 5000
    a = rng.integers(0, 50, n).astype(np.int32)      # 50 distinct
    b = rng.integers(0, 5, n).astype(np.int32)       # 5 distinct: sorted on first
    x = rng.standard_normal(n)
    rel = Relation('R', [Column('a', 'key', a), Column('b', 'key', b), Column('x', 'cont', x)])
    s = sort_by_join_attributes(rel, ['a', 'b'])
    sa, sb, sx = (s.col(c).data for c in 'abx')
    key = sb.astype(np.int64) * 100 + sa
    assert np.all(np.diff(key) >= 0)
    before = sorted(zip(a.tolist(), b.tolist(), x.tolist()))
    after = sorted(zip(sa.tolist(), sb.tolist(), sx.tolist()))
    assert before == after


def _lex_sorted(cols):
    """Rows non-decreasing in the lexicographic order of cols (first most significant)."""
    idx = np.lexsort(list(reversed(cols)))
    return all(np.array_equal(c[idx], c) for c in cols)


def test_config1_recipe():
    sch, batch = config1(20_000)
    R, S, T = sch.rel('R'), sch.rel('S'), sch.rel('T')
    assert (R.nrows, S.nrows, T.nrows) == (20_000, 1000, 500)
    assert np.array_equal(S.col('k1').data, np.arange(1000))
    assert np.array_equal(T.col('k2').data, np.arange(500))
    assert all(R.col(f'r{i}').data.dtype == np.float64 for i in range(3))
    assert len(batch) == 66
    assert _lex_sorted([R.col('k2').data, R.col('k1').data])   # 500 distinct before 1000


def test_config2_recipe():
    n = 300_000
    sch, batch = config2(n)
    F = sch.rel('F')
    sizes = {r.name: r.nrows for r in sch.relations}
    assert sizes == {'F': n, 'D1': 100_000, 'Sub1': 5000, 'Sub2': 500, 'D2': 10_000,
                     'D3': 1000, 'D4': 1000}
    for p, c, k in sch.edges:
        K = sch.rel(c).nrows
        assert np.array_equal(sch.rel(c).col(k).data, np.arange(K))    # dense unique keys
        fk = sch.rel(p).col(k).data
        assert fk.min() >= 0 and fk.max() < K
    assert [f for f in sch.meta['features'] if f.startswith('x')] == [f'x{i}' for i in range(8)]
    assert len(sch.meta['features']) == 30 and len(sch.meta['cats']) == 10
    assert len(batch) == 851
    for f in [f'x{i}' for i in range(8)]:
        assert F.col(f).data.dtype == np.float32
    # fact rows in the scan order of Sec. 3.5: (k3, k2, k1), fewest distinct first
    assert _lex_sorted([F.col('k3').data, F.col('k2').data, F.col('k1').data])
    # categories over log-uniform domains in [5, 1000], values inside them
    for r in sch.relations:
        for c in r.columns:
            if c.role == 'cat':
                assert 5 <= c.cat_domain <= 1000
                assert c.data.min() >= 0 and c.data.max() < c.cat_domain
    # foreign keys Zipf 0.8 (the 100k-key k1 is too sparse at this size for a slope)
    assert abs(_rank_slope(F.col('k3').data, 1000, top=50) + 0.8) < 0.1
    # features: even-numbered N(0,1), odd-numbered the LogNormal mixture (mean 3.01)
    x0, x1 = F.col('x0').data.astype(np.float64), F.col('x1').data.astype(np.float64)
    assert abs(x0.mean()) < 0.02 and abs(x0.std() - 1) < 0.02
    mix_mean = 0.7 * np.exp(0.125) + 0.3 * np.exp(2.0)
    assert x1.min() > 0 and abs(x1.mean() / mix_mean - 1) < 0.03


def test_config2_orders_hold_the_same_rows_and_seeds_repeat():
    a, _ = config2(20_000)
    b, _ = config2(20_000, fact_order='random')
    ka = np.stack([a.rel('F').col(k).data for k in ('k1', 'k2', 'k3')], 1)
    kb = np.stack([b.rel('F').col(k).data for k in ('k1', 'k2', 'k3')], 1)
    assert not np.array_equal(ka, kb)
    assert np.array_equal(ka[np.lexsort(ka.T)], kb[np.lexsort(kb.T)])
    for ra, rb in zip(a.relations[1:], b.relations[1:]):            # same dimensions
        for ca, cb in zip(ra.columns, rb.columns):
            assert np.array_equal(ca.data, cb.data)
    c, _ = config2(20_000)
    assert all(np.array_equal(x.data, y.data) for x, y in zip(a.rel('F').columns, c.rel('F').columns))
    with pytest.raises(ValueError):
        config2(10, fact_order='shuffled')


def test_config3_recipe():
    sch, batch = config3(100_000, sample_rows=100_000)
    feats, thr, nodes = sch.meta['features'], sch.meta['thresholds'], sch.meta['nodes']
    assert len(feats) == 20 and len(nodes) == 64
    assert all(len(n) == 6 for n in nodes)
    for f in feats:
        t = thr[f]
        assert 1 <= len(t) <= 32 and np.all(np.diff(t) > 0)
        assert np.array_equal(t.astype(np.float32).astype(np.float64), t)   # FP32-exact
    assert len(batch) == 64 * sum(len(thr[f]) for f in feats) * 3
    assert sch.rel('F').col('y').data.dtype == np.float32


def test_config3_classification_recipe():
    sch, batch = config3_classification(100_000, n_classes=4, sample_rows=100_000)
    feats, thr, nodes = sch.meta['features'], sch.meta['thresholds'], sch.meta['nodes']
    assert len(feats) == 20 and len(nodes) == 64 and sch.meta['n_classes'] == 4
    cls = sch.rel('F').col('cls')
    assert cls.role == 'cat' and cls.cat_domain == 4 and cls.data.dtype == np.int32
    share = np.bincount(cls.data, minlength=4) / len(cls.data)
    assert np.all(np.abs(share - 0.25) < 0.01)                          # quantile bins of the score
    assert 'y' not in sch.rel('F').names()
    for f in feats:
        assert np.array_equal(thr[f].astype(np.float32).astype(np.float64), thr[f])
    # per node: its two queries, then two per (feature, threshold)
    assert len(batch) == 64 * (2 + 2 * sum(len(thr[f]) for f in feats))
    assert batch[0].group_by == ('cls',) and batch[1].group_by == () and batch[0].factors == nodes[0]
    assert batch[2].factors == nodes[0] + ((feats[0], 'le', float(thr[feats[0]][0])),)
    # the seed repeats its data
    sch2, batch2 = config3_classification(100_000, n_classes=4, sample_rows=100_000)
    assert np.array_equal(sch2.rel('F').col('cls').data, cls.data) and batch2 == batch


def test_many_to_many_recipe():
    sch, batch = many_to_many(50_000, n_user=5_000, n_business=1_000, seed=2)
    assert [r.name for r in sch.relations] == ['Review', 'User', 'Business', 'Category', 'Attribute']
    R, C, A = sch.rel('Review'), sch.rel('Category'), sch.rel('Attribute')
    assert R.nrows == 50_000 and sch.rel('User').nrows == 5_000 and sch.rel('Business').nrows == 1_000
    nc = np.bincount(C.col('business_id').data, minlength=1_000)
    na = np.bincount(A.col('business_id').data, minlength=1_000)
    assert nc.min() >= 1 and nc.max() <= 8 and na.min() == 0 and na.max() <= 12
    assert np.all(np.diff(C.col('business_id').data) >= 0) and C.col('cat').data.max() < 40
    assert 0 <= R.col('user_id').data.min() and R.col('user_id').data.max() < 5_000
    assert set(np.unique(R.col('stars').data)) <= {1.0, 2.0, 3.0, 4.0, 5.0}
    assert len(batch) == 45 + 1 and batch[-1].group_by == ('cat',)
    # sorted on the join attributes (fewest distinct values first: business, then user),
    # and the random order holds the same rows
    order = np.lexsort([R.col('user_id').data, R.col('business_id').data])
    assert np.array_equal(order, np.arange(R.nrows))
    rnd, _ = many_to_many(50_000, n_user=5_000, n_business=1_000, seed=2, fact_order='random')
    for c in R.names():
        assert np.array_equal(np.sort(R.col(c).data), np.sort(rnd.rel('Review').col(c).data))


def test_config4_recipe():
    n = 200_000
    sch, batch = config4(n)
    F = sch.rel('F')
    assert [sch.rel(f'D{j}').nrows for j in range(1, 5)] == [200, 1000, 5000, 20000]
    ncat = [sum(c.role == 'cat' for c in sch.rel(f'D{j}').columns) for j in range(1, 5)]
    assert ncat == [7, 7, 8, 8] and len(sch.meta['cats']) == 30
    assert [sch.rel(f'D{j}').col(f'd{j}_c0').cat_domain for j in (1, 2, 3)] == [50, 20, 10]
    assert sch.meta['cube'] == ['d1_c0', 'd2_c0', 'd3_c0']
    assert len(batch) == 435 + 30 + 8 == 473
    assert _lex_sorted([F.col(f'k{j}').data for j in range(1, 5)])
    assert abs(_rank_slope(F.col('k2').data, 1000, top=50) + 1.0) < 0.1


@pytest.mark.parametrize('index', list(range(0, 500, 25)))
def test_config5_recipe(index):
    sch, batch = config5_schema(index, n_scale=1e-3)
    n = len(sch.relations)
    assert 3 <= n <= 8 and len(sch.edges) == n - 1
    children = [c for _, c, _ in sch.edges]
    assert len(set(children)) == n - 1 and sch.root not in children     # a tree
    assert 0.0 <= sch.meta['skew'] <= 1.2
    real = [f for f in sch.meta['features'] if not f.startswith('f_pad')]
    assert 5 <= len(real) <= 40
    assert 10 <= sum(not a.group_by for a in batch) <= 2000
    for p, c, k in sch.edges:
        fk = sch.rel(p).col(k).data
        assert fk.min() >= 0 and fk.max() < sch.rel(c).nrows
    fact_fks = [sch.rel('F').col(k).data for p, _, k in sch.edges if p == 'F']
    if index % 2 == 0 and fact_fks:    # even indices: the fact sorted on its join attributes
        assert any(np.all(np.diff(fk) >= 0) for fk in fact_fks)
