"""Plans rooted at any relation (Sec. 3.2 directional views, Sec. 3.3 root
choice): reversed edges turn a parent's foreign key into the child key, the
fact table becomes a fanning-out view, and every plan gives the oracle's
results.  View merging off gives the same results too."""
import numpy as np
import pytest

from oracle import oracle
from workloads import config1, config2, covar_batch, tiny_schema

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu


def _run(sch, batch, **kw):
    from paper_1906_08687_gb300 import Engine, register_schema
    from lmf_testlib import to_device
    eng = Engine(0)
    tens = to_device(sch)
    register_schema(eng, sch, tens)
    bid = eng.declare_batch(batch)
    eng.plan(bid, **kw)
    eng.run(bid)
    eng.sync(bid)
    out = eng.results(bid, len(batch))
    info = eng.plan_info(bid)
    eng.close()
    return out, info


@pytest.mark.parametrize('root', ['S', 'T'])
def test_config1_rooted_at_a_dimension(root):
    sch, batch = config1(50_000)
    rid = [r.name for r in sch.relations].index(root)
    got, info = _run(sch, batch, precision=0, batching=0, root_mode=1, root_rel=rid)
    assert info['root_rel'] == rid and info['unique_keys'] == 0
    fails, stats = compare(got, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:3], stats)


@pytest.mark.parametrize('seed', list(range(10)))
def test_tiny_every_root(seed):
    sch, _ = tiny_schema(9100 + seed)
    batch = covar_batch(sch.meta['features'])
    want = oracle.evaluate(sch, batch)
    from paper_1906_08687_gb300 import LmfError
    for rid in range(len(sch.relations)):
        try:
            got, info = _run(sch, batch, precision=0, batching=0, root_mode=1, root_rel=rid)
        except LmfError as e:
            assert e.status == -10      # an irreversible (sparse) key edge
            continue
        fails, stats = compare(got, want, arith_floor=ARITH_FLOOR)
        assert not fails, (rid, fails[:3], stats)


def test_merge_off_same_results():
    sch, batch = config2(300_000)
    a, ia = _run(sch, batch, precision=1, batching=1)
    b, ib = _run(sch, batch, precision=1, batching=1, no_merge=1)
    assert ia['merged'] == 1 and ib['merged'] == 0 and ib['n_probe_groups'] == 4
    for x, y in zip(a, b):
        if x.dtype == np.int64:
            assert np.array_equal(x, y)
    fails, _ = compare(b, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails


def test_heuristic_root_rule():
    """Ungrouped batch: every relation has equal weight, the largest wins."""
    sch, batch = config1(20_000)
    got, info = _run(sch, batch, precision=0, batching=0, root_mode=2)
    assert info['root_rel'] == 0
    fails, _ = compare(got, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails


# ----------------------------------------------------------------------------
# per-query roots (LMF_ROOT_PER_QUERY)
def test_chain_each_query_at_its_own_root():
    """Sec. 3.3's chain S_1 ... S_{n-1} (many-to-many joins): Q_i = COUNT grouped
    by X_i for every i.  From the declared root S_1 only Q_1 evaluates (X_2.. sit
    behind fanning-out keys); with per-query roots each Q_i runs at a root
    holding X_i and every count is bit-identical to the oracle's (the L_i R_i
    products)."""
    from workloads import Agg, chain_schema
    n, size, dom = 6, 400, 7
    sch = chain_schema(n, size, dom, seed=3, group_copies=True)
    batch = [Agg(group_by=('X1',))] + [Agg(group_by=(f'G{i}',)) for i in range(2, n)] + [Agg(group_by=(f'X{n}',))]
    want = oracle.evaluate(sch, batch)
    got, info = _run(sch, batch, precision=0, batching=1, root_mode=3)
    assert info['n_roots'] >= n - 1
    for i, (g, w) in enumerate(zip(got, want.values)):
        assert np.array_equal(np.asarray(g, np.int64), w), i
    # the same batch from the declared root alone is refused
    from paper_1906_08687_gb300 import LmfError
    with pytest.raises(LmfError):
        _run(sch, batch, precision=0, batching=1, root_mode=0)


@pytest.mark.parametrize('seed', [0, 1, 3, 4, 6, 7])
def test_tiny_fanout_grouped_per_query(seed):
    """Tiny schemas with duplicate child keys and dangling foreign keys: the
    covar batch plus COUNT and SUM(x) grouped by every category, categories
    behind fanning-out keys included, evaluated with per-query roots, against
    the oracle (counts bit-exact, sums within the error rule with the small-input
    floor); twice in a row (the per-root plans and the result copies repeat)."""
    from workloads import grouped_batch
    sch, _ = tiny_schema(5000 + seed, unique_keys=False)
    feats, cats = sch.meta['features'], sch.meta['cats']
    batch = covar_batch(feats) + grouped_batch(cats, feats)
    want = oracle.evaluate(sch, batch)
    from paper_1906_08687_gb300 import Engine, register_schema
    from lmf_testlib import to_device
    eng = Engine(0)
    tens = to_device(sch)
    register_schema(eng, sch, tens)
    bid = eng.declare_batch(batch)
    eng.plan(bid, precision=0, batching=1, root_mode=3)
    for _ in range(2):
        eng.run(bid)
        eng.sync(bid)
        got = eng.results(bid, len(batch))
        fails, stats = compare(got, want, arith_floor=ARITH_FLOOR)
        assert not fails, (fails[:3], stats, eng.plan_info(bid))
    eng.close()


def test_per_query_keeps_a_batch_that_fits_the_declared_root():
    """A batch the declared root evaluates is planned there as one plan."""
    sch, batch = config1(20_000)
    got, info = _run(sch, batch, precision=0, batching=1, root_mode=3)
    assert info['n_roots'] == 1 and info['root_rel'] == 0
    fails, stats = compare(got, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:3], stats)
