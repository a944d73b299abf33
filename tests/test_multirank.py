"""The N > 1 host path of bench.py on CPU: two gloo ranks.

Every rank runs its own seeded instance (weak scaling, no collective on the
data path); the step time is the maximum over ranks and rank 0 reports the
whole job.  Checked here without a GPU: the max-over-ranks reduction, the
barrier, and that the ranks' instances differ (seed + 1000 * rank) while
having the same shape."""
import argparse
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group('gloo', rank=rank, world_size=ws)
    import bench
    assert bench.dist_env()[:2] == (ws, rank)
    t = bench.max_over_ranks(ws, 1.5 * (rank + 1))
    bench.barrier(ws)
    args = argparse.Namespace(gen='config1', cfg_index=1, n_fact=2000, fact_order='sorted')
    sch, batch = bench.make_workload(args, rank)
    x = sch.rel(sch.root).col('r0').data
    np.save(os.path.join(out_dir, f'r{rank}.npy'), np.concatenate([[t, len(batch)], x[:50]]))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks(tmp_path):
    ws = 2
    mp.spawn(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r0, r1 = (np.load(tmp_path / f'r{r}.npy') for r in range(ws))
    assert r0[0] == r1[0] == 3.0                 # max over ranks of 1.5, 3.0
    assert r0[1] == r1[1] == 66                  # same batch on every rank
    assert not np.array_equal(r0[2:], r1[2:])    # different seeded instances


def _shard_rank(rank, ws, port, out_dir):
    """One rank of the sharded exchange: the oracle evaluates the batch over this
    rank's root rows (standing in for the engine, which needs a GPU), the packed
    results are summed over the ranks with one gloo all-reduce per array, and
    rank 0 saves the combined results."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group('gloo', rank=rank, world_size=ws)
    from oracle import oracle
    from paper_1906_08687_gb300 import shard
    from workloads import config2
    sch, batch = config2(20_011)
    n = sch.rel(sch.root).nrows
    b, e = shard.row_range(n, rank, ws)
    part = oracle.evaluate(shard.shard_schema(sch, b, e), batch)
    i64, f64 = shard.pack(part.values, sch, batch)
    ti, tf = torch.from_numpy(i64), torch.from_numpy(f64)
    shard.allreduce_packed(ti, tf, dist.all_reduce)
    if rank == 0:
        np.save(os.path.join(out_dir, 'i64.npy'), ti.numpy())
        np.save(os.path.join(out_dir, 'f64.npy'), tf.numpy())
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_sharded_exchange_two_gloo_ranks(tmp_path):
    """Row ranges of the root on two ranks + one all-reduce of the packed
    partials = the batch over the whole join: counts bit for bit, sums within
    the error rule (FP64 partials, rounding order only)."""
    from oracle import oracle
    from oracle.compare import compare
    from paper_1906_08687_gb300 import shard
    from workloads import config2
    ws = 2
    mp.spawn(_shard_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    sch, batch = config2(20_011)
    got = shard.unpack(np.load(tmp_path / 'i64.npy'), np.load(tmp_path / 'f64.npy'), sch, batch)
    want = oracle.evaluate(sch, batch)
    fails, stats = compare(got, want)
    assert not fails, (fails[:3], stats)
    assert stats['max_err_over_allowed'] < 1e-3      # FP64 partials: only the summation order differs


def test_row_ranges_partition_the_root():
    from paper_1906_08687_gb300 import shard
    for n in (0, 1, 7, 1000, 20_000_003):
        for ws in (1, 2, 3, 8):
            rr = [shard.row_range(n, r, ws) for r in range(ws)]
            assert rr[0][0] == 0 and rr[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
            assert max(e - b for b, e in rr) - min(e - b for b, e in rr) <= 1
    with pytest.raises(ValueError):
        shard.row_range(10, 2, 2)


def test_pack_unpack_layout():
    """The packed layout: counts in the int64 array and sums in the float64 array,
    each in aggregate order, grouped cells row-major; unpack inverts pack."""
    from paper_1906_08687_gb300 import shard
    from workloads import config2
    sch, batch = config2(1000)
    layout, n_i, n_f = shard.result_layout(sch, batch)
    assert n_i == sum(n for c, n, _ in layout if c) and n_f == sum(n for c, n, _ in layout if not c)
    rng = np.random.default_rng(3)
    vals = [(rng.integers(0, 99, n) if c else rng.standard_normal(n)) for c, n, _ in layout]
    i64, f64 = shard.pack(vals, sch, batch)
    back = shard.unpack(i64, f64, sch, batch)
    assert all(np.array_equal(a, b) for a, b in zip(vals, back))
    assert layout[0] == (True, 1, 0)                  # COUNT first
    assert layout[1] == (False, 1, 0)                 # SUM(x0): the first float cell
