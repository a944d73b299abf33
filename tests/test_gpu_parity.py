"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Counts bit-exact, sums within the error rule of lmf_testlib (1e-6 relative,
floor 1e-3 of the sum of absolute values).
"""
import numpy as np
import pytest

from oracle import oracle
from workloads import Agg, config1, config2, covar_batch, grouped_batch, tiny_schema

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu

PLAIN, SPLIT = 0, 1
SINGLE, GRAPH = 0, 1


def _check(sch, batch, precision=PLAIN, batching=SINGLE, floor=0.0, **kw):
    got, info, eng = run_engine(sch, batch, precision=precision, batching=batching, **kw)
    want = oracle.evaluate(sch, batch)
    fails, stats = compare(got, want, arith_floor=floor)
    assert not fails, (fails[:5], stats, info)
    eng.close()
    return got, info, stats


@pytest.mark.parametrize('precision', [PLAIN, SPLIT])
@pytest.mark.parametrize('batching', [SINGLE, GRAPH])
def test_config1_star_full(precision, batching):
    sch, batch = config1()
    _, info, stats = _check(sch, batch, precision, batching)
    assert info['n_gram_aggs'] == 65 and info['z_len'] == 11
    assert info['precision'] == precision     # SPLIT runs on the tcgen05 kernel


def test_config1_ragged_sizes():
    for n in [1, 255, 257, 12345, 100003]:
        sch, batch = config1(n)
        _check(sch, batch, PLAIN, SINGLE, floor=ARITH_FLOOR)


@pytest.mark.parametrize('precision', [PLAIN, SPLIT])
def test_config2_snowflake_reduced(precision):
    sch, batch = config2(300_007)
    _, info, stats = _check(sch, batch, precision, GRAPH, floor=ARITH_FLOOR)
    assert info['precision'] == precision
    assert info['n_grouped_aggs'] == 10 * 31 + 45
    assert info['n_views'] == 6 and info['n_probe_groups'] == 3


def test_empty_root():
    sch, batch = config1(0)
    got, info, eng = run_engine(sch, batch, precision=PLAIN, batching=SINGLE)
    assert got[0][0] == 0
    assert all(np.all(g == 0) for g in got)
    eng.close()


@pytest.mark.parametrize('seed', list(range(24)))
def test_tiny_schemas_fanout_dangling(seed):
    """Duplicate child keys (joins fan out), dangling foreign keys, empty
    relations.  Grouped aggregates only where every key is unique."""
    uniq = seed % 3 == 2
    sch, _ = tiny_schema(5000 + seed, unique_keys=uniq)
    feats, cats = sch.meta['features'], sch.meta['cats']
    batch = covar_batch(feats)
    if uniq:
        batch += grouped_batch(cats, feats)
    _check(sch, batch, PLAIN if seed % 2 else SPLIT, SINGLE, floor=ARITH_FLOOR)


def test_deterministic_runs():
    sch, batch = config2(200_000)
    outs, _, eng = run_engine(sch, batch, precision=PLAIN, batching=GRAPH, runs=3)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    eng.close()


def test_unsupported_shapes_fail_cleanly():
    from paper_1906_08687_gb300 import LmfError
    sch, _ = config1(1000)
    bad = [Agg(factors=(('r0', 'pow', 2), ('r1', 'pow', 1)))]   # degree 3
    with pytest.raises(LmfError) as e:
        run_engine(sch, bad)
    assert e.value.status == -10
