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
