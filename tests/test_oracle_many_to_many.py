"""Pins for the oracle on a many-to-many join much larger than its inputs
(workloads.many_to_many, the Yelp shape of Sec. 4: a review joins with every
category and every attribute row of its business).

* A tiny instance against the brute-force natural join (Cartesian product).
* A 20k-review instance (a join some tens of times larger than the inputs)
  against every aggregate of its batch evaluated in factorised form by hand:
  a review's tuples are the cross product of its business's category and
  attribute rows, so SUM(prod) over the join is, per review, the product of
  the review-side factors, the sum over the business's category rows of the
  category factors and the sum over its attribute rows of the attribute
  factors (the distributivity of Sec. 1.1 written out per aggregate).
"""
import numpy as np
import pytest

from oracle import oracle
from oracle_pinlib import check_against_brute_force
from workloads import many_to_many

SIDE = {'stars': 'Review', 'useful': 'Review', 'fans': 'User', 'review_count': 'User',
        'bstars': 'Business', 'lat': 'Business', 'cat_w': 'Category', 'attr_val': 'Attribute'}


def test_tiny_instance_matches_brute_force():
    for seed in range(4):
        sch, batch = many_to_many(7, n_user=3, n_business=3, max_categories=2, max_attributes=2, seed=seed)
        check_against_brute_force(sch, batch)


def _factorised(sch, agg):
    """Per-review value of the aggregate over its join tuples, and of
    SUM(|value|), written out from the relations (float64 numpy)."""
    R, U, B = sch.rel('Review'), sch.rel('User'), sch.rel('Business')
    C, A = sch.rel('Category'), sch.rel('Attribute')
    nb = B.nrows
    u = R.col('user_id').data
    b = R.col('business_id').data
    row = np.ones(R.nrows)
    cat_f = np.ones(C.nrows)
    att_f = np.ones(A.nrows)
    for attr, kind, p in agg.factors:
        assert kind == 'pow'
        side = SIDE[attr]
        if side == 'Review':
            row = row * R.col(attr).data.astype(np.float64) ** int(p)
        elif side == 'User':
            row = row * U.col(attr).data.astype(np.float64)[u] ** int(p)
        elif side == 'Business':
            row = row * B.col(attr).data.astype(np.float64)[b] ** int(p)
        elif side == 'Category':
            cat_f = cat_f * C.col(attr).data.astype(np.float64) ** int(p)
        else:
            att_f = att_f * A.col(attr).data.astype(np.float64) ** int(p)
    cb, ab = C.col('business_id').data, A.col('business_id').data
    sc = np.bincount(cb, weights=cat_f, minlength=nb)
    sa = np.bincount(ab, weights=att_f, minlength=nb)
    sc_abs = np.bincount(cb, weights=np.abs(cat_f), minlength=nb)
    sa_abs = np.bincount(ab, weights=np.abs(att_f), minlength=nb)
    return row * sc[b] * sa[b], np.abs(row) * sc_abs[b] * sa_abs[b]


def test_covar_and_grouped_counts_in_factorised_form():
    sch, batch = many_to_many(20_000, n_user=2_000, n_business=500, seed=3)
    res = oracle.evaluate(sch, batch)
    R, C, A = sch.rel('Review'), sch.rel('Category'), sch.rel('Attribute')
    b = R.col('business_id').data
    nc = np.bincount(C.col('business_id').data, minlength=500)
    na = np.bincount(A.col('business_id').data, minlength=500)
    join = int(np.sum(nc[b].astype(np.int64) * na[b]))
    assert res.join_size == join
    inputs = sum(r.nrows for r in sch.relations)
    assert join > 10 * inputs                      # the join is much larger than its inputs
    for a, agg in enumerate(batch):
        if agg.group_by:
            # COUNT by cat: per review, its business's attribute rows times its category rows of value k
            H = np.zeros((500, 40), np.int64)
            np.add.at(H, (C.col('business_id').data, C.col('cat').data), 1)
            want = (H[b] * na[b][:, None]).sum(axis=0)
            np.testing.assert_array_equal(np.asarray(res.values[a], np.int64), want)
            continue
        per_review, per_review_abs = _factorised(sch, agg)
        if not agg.factors:
            assert int(res.values[a][0]) == join
            continue
        want, scale = float(np.sum(per_review)), float(np.sum(per_review_abs))
        got = float(np.asarray(res.values[a]).reshape(-1)[0])
        assert abs(got - want) <= 1e-12 * scale, (agg, got, want, scale)
        assert abs(float(np.asarray(res.abs[a]).reshape(-1)[0]) - scale) <= 1e-12 * scale


@pytest.mark.parametrize('order', ['sorted', 'random'])
def test_input_order_keeps_the_values(order):
    sch, batch = many_to_many(3_000, n_user=300, n_business=100, seed=9, fact_order=order)
    ref, _ = many_to_many(3_000, n_user=300, n_business=100, seed=9, fact_order='sorted')
    got, want = oracle.evaluate(sch, batch), oracle.evaluate(ref, batch)
    assert got.join_size == want.join_size
    for a in range(len(batch)):
        if got.kinds[a] == 'count':
            assert np.array_equal(got.values[a], want.values[a])
        else:
            g, w = float(np.asarray(got.values[a]).reshape(-1)[0]), float(np.asarray(want.values[a]).reshape(-1)[0])
            assert abs(g - w) <= 1e-12 * float(np.asarray(want.abs[a]).reshape(-1)[0])
