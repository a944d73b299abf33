"""Sharding of the root by row ranges (paper_1906_08687_gb300.shard), emulated
on one GPU: every shard registers its slice of the root's device columns (the
same memory, offset pointers) with the dimensions whole, runs the whole batch,
and exports its packed results to device buffers; the exchange a multi-GPU
run does with one all-reduce per array is emulated by summing the shards'
device buffers.  The sum equals the unsharded run -- counts bit for bit, sums
within the error rule against the oracle -- and the host-side result layout
equals the engine's."""
import numpy as np
import pytest

from oracle import oracle
from workloads import config2, config4, to_device

from lmf_testlib import ARITH_FLOOR, compare

pytestmark = pytest.mark.gpu


def _packed_run(sch, batch, tensors):
    import torch
    from paper_1906_08687_gb300 import Engine, register_schema
    eng = Engine(0)
    register_schema(eng, sch, tensors)
    bid = eng.declare_batch(batch)
    eng.plan(bid, precision=0, batching=1)
    eng.run(bid)
    eng.sync(bid)
    n_i, n_f = eng.result_sizes(bid)
    i64 = torch.zeros(max(1, n_i), dtype=torch.int64, device='cuda')
    f64 = torch.zeros(max(1, n_f), dtype=torch.float64, device='cuda')
    eng.read_results(bid, i64.data_ptr(), f64.data_ptr(), True)
    torch.cuda.synchronize()
    layout = eng.result_layout(bid, len(batch))
    eng.close()
    return i64[:n_i], f64[:n_f], layout


@pytest.mark.parametrize('make,world', [(lambda: config2(300_007), 3), (lambda: config4(200_001), 4)])
def test_root_partition_sums_to_whole(make, world):
    from paper_1906_08687_gb300 import shard
    sch, batch = make()
    dev = to_device(sch)
    n = sch.rel(sch.root).nrows
    wi, wf, layout = _packed_run(sch, batch, dev)
    mine, n_i, n_f = shard.result_layout(sch, batch)
    assert n_i == wi.numel() and n_f == wf.numel()
    assert [(n, off) for _, n, off in mine] == [(n, off) for n, _, off in layout]
    si, sf = None, None
    for r in range(world):
        b, e = shard.row_range(n, r, world)
        pi, pf, _ = _packed_run(shard.shard_schema(sch, b, e), batch, shard.shard_tensors(sch, dev, b, e))
        si = pi if si is None else si + pi         # the all-reduce (sum), emulated
        sf = pf if sf is None else sf + pf
    assert np.array_equal(si.cpu().numpy(), wi.cpu().numpy())      # counts bit for bit
    got = shard.unpack(si.cpu().numpy(), sf.cpu().numpy(), sch, batch)
    want = oracle.evaluate(sch, batch)
    fails, stats = compare(got, want, arith_floor=ARITH_FLOOR)
    assert not fails, (fails[:3], stats)
