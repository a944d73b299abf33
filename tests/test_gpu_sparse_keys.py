"""Join keys too sparse for direct addressing (the key index of A1): the
engine renumbers them by rank among the distinct child keys, and every
aggregate matches the oracle, which joins on the original values."""
import numpy as np
import pytest

from oracle import oracle
from workloads import config2, covar_batch, grouped_batch, spread_keys, tiny_schema

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('seed', list(range(8)))
def test_tiny_sparse_keys(seed):
    """Duplicate and dangling keys, empty relations, keys ~1e6 apart."""
    uniq = seed % 3 == 2
    sch, _ = tiny_schema(5000 + seed, unique_keys=uniq)
    sp = spread_keys(sch)
    feats, cats = sch.meta['features'], sch.meta['cats']
    batch = covar_batch(feats) + (grouped_batch(cats, feats) if uniq else [])
    got, info, eng = run_engine(sp, batch, precision=0, batching=0)
    fails, stats = compare(got, oracle.evaluate(sp, batch), arith_floor=ARITH_FLOOR)
    eng.close()
    assert not fails, (fails[:5], stats, info)


def test_config2_sparse_keys_match_dense_keys():
    """Every join attribute of the snowflake spread 10^4 apart (up to ~1e9):
    the same counts bit for bit as the dense-key run, sums within the rule."""
    sch, batch = config2(100_000)
    sp = spread_keys(sch, mult=10_000)
    got, info, eng = run_engine(sp, batch, precision=0, batching=1)
    eng.close()
    dense, _, eng2 = run_engine(sch, batch, precision=0, batching=1)
    eng2.close()
    fails, stats = compare(got, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:5], stats, info)
    for g, d in zip(got, dense):
        if np.asarray(g).dtype == np.int64:
            assert np.array_equal(g, d)
