"""Property-based pins for the oracle (hypothesis): random batches on random
tiny schemas (fan-out, dangling keys, empty relations) against the
brute-force natural join, and identities every aggregate satisfies whatever
the data:

* summed over its groups, a grouped aggregate is the ungrouped one (Sec. 2:
  a group-by partitions the join);
* 1[x <= t] + 1[x > t] = 1, so the two halves of a threshold add up to the
  aggregate without it (the Kronecker deltas of Sec. 1.1).
"""
import numpy as np
import pytest

from oracle import oracle
from oracle_pinlib import assert_close, check_against_brute_force
from workloads import Agg, tiny_schema

hyp = pytest.importorskip('hypothesis')
st = pytest.importorskip('hypothesis.strategies')
given, settings = hyp.given, hyp.settings


@st.composite
def schema_and_batch(draw):
    seed = draw(st.integers(0, 2**31 - 1))
    sch, _ = tiny_schema(seed, max_rows=8, allow_empty=draw(st.sampled_from([False, False, True])),
                         unique_keys=draw(st.sampled_from([False, False, True])))
    feats, cats = sch.meta['features'], sch.meta['cats']
    batch = []
    for _ in range(draw(st.integers(1, 6))):
        gb = tuple(draw(st.lists(st.sampled_from(cats), max_size=2, unique=True))) if cats else ()
        factors = []
        for _ in range(draw(st.integers(0, 3))):
            f = draw(st.sampled_from(feats))
            kind = draw(st.sampled_from(['pow', 'le', 'gt']))
            if kind == 'pow':
                factors.append((f, 'pow', draw(st.sampled_from([1, 2]))))
            else:
                col = sch.owner(f).col(f).data
                t = float(draw(st.sampled_from(list(col)))) if len(col) else 0.0
                factors.append((f, kind, t + draw(st.sampled_from([0.0, -0.5, 0.25]))))
        batch.append(Agg(group_by=gb, factors=tuple(factors)))
    return sch, batch


@settings(max_examples=80, deadline=None)
@given(schema_and_batch())
def test_random_batches_match_brute_force(sb):
    sch, batch = sb
    check_against_brute_force(sch, batch)


@settings(max_examples=60, deadline=None)
@given(schema_and_batch(), st.data())
def test_groups_and_threshold_halves_add_up(sb, data):
    sch, batch = sb
    agg = batch[0]
    feats = sch.meta['features']
    f = data.draw(st.sampled_from(feats))
    col = sch.owner(f).col(f).data
    t = float(np.median(col)) if len(col) else 0.0
    ungrouped = Agg(factors=agg.factors)
    le = Agg(group_by=agg.group_by, factors=agg.factors + ((f, 'le', t),))
    gt = Agg(group_by=agg.group_by, factors=agg.factors + ((f, 'gt', t),))
    whole = Agg(group_by=agg.group_by, factors=agg.factors)
    res = oracle.evaluate(sch, [ungrouped, whole, le, gt])
    v = [np.asarray(x) for x in res.values]
    if res.kinds[0] == 'count':
        assert int(v[1].sum()) == int(v[0].sum())
        assert np.array_equal(v[2] + v[3], v[1])
    else:
        scale = float(np.sum(res.abs[1])) + 1e-300
        assert abs(float(v[1].sum()) - float(v[0].sum())) <= 1e-12 * scale
        assert_close(v[2] + v[3], v[1], rel=1e-12, absolute=1e-12 * scale)
