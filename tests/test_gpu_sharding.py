"""Sharding of the root by row ranges, emulated on one GPU: every shard runs
the whole batch over its rows (dimensions replicated), the partial results
are summed on the host (int64 counts exactly, FP64 sums), and the sum equals
the unsharded run -- counts bit for bit, sums within the error rule against
the oracle.  This is the exchange a multi-GPU run would do with one
all-reduce, emulated on one GPU."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle
from workloads import Relation, Schema, config2, config4

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu


def _shard(sch, lo, hi):
    root = sch.rel(sch.root)
    part = Relation(root.name, [dataclasses.replace(c, data=np.ascontiguousarray(c.data[lo:hi]))
                                for c in root.columns])
    rels = [part if r.name == sch.root else r for r in sch.relations]
    return Schema(rels, sch.edges, sch.root, dict(sch.meta))


@pytest.mark.parametrize('make,bounds', [
    (lambda: config2(300_007), [0, 100_000, 200_003, 300_007]),
    (lambda: config4(200_001), [0, 1, 77_777, 200_001]),
])
def test_root_partition_sums_to_whole(make, bounds):
    sch, batch = make()
    whole, _, e0 = run_engine(sch, batch, precision=0, batching=1)
    e0.close()
    parts = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        got, _, e = run_engine(_shard(sch, lo, hi), batch, precision=0, batching=1)
        parts.append(got)
        e.close()
    want = oracle.evaluate(sch, batch)
    summed = []
    for i in range(len(batch)):
        s = sum(np.asarray(p[i]) for p in parts)
        if want.kinds[i] == 'count':
            assert np.array_equal(s.astype(np.int64), np.asarray(whole[i]).astype(np.int64)), batch[i]
        summed.append(s)
    fails, stats = compare(summed, want, arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:3], stats)
