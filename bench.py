#!/usr/bin/env python3
"""Benchmark of one aggregate batch over a snowflake join (config 2 shape).

Workload: fact table of 20M rows (3 int32 foreign keys, 8 FP32 features)
joined to a 3-level snowflake of 6 dimension relations (22 more continuous
features, 10 categorical attributes); the batch is COUNT, all 495 degree <= 2
monomial SUMs over the 30 features, SUM(x_i) and COUNT grouped by each
categorical attribute, and COUNT grouped by every categorical pair: 851
aggregates (Sec. 2, covar matrix with one-hot categorical group-bys).

A step is one lmf_run of the whole batch (child views, root scan, combine,
placement) with the inputs resident in HBM.  Metric: joined tuples x
aggregates / step time, in G joined-tuple-aggregates/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload snowflake|tree|chowliu|star]

The default workload is the snowflake batch above; --workload selects the
other batches of the same engine (the regression-tree level batch, the
Chow-Liu pair counts with a data cube, the star covar batch) at their own
sizes, reported in the same JSON form.

Under torchrun (N > 1) every rank runs its own seeded instance (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'G joined-tuple-aggregates/s, HBM % of peak; speedup vs plain at ≤1e-6 rel err'
UNIT = 'G joined-tuple-aggregates/s'
# workload -> (generator, config index, fact rows, CPU-baseline rows, reference-arm rows per step,
# aggregates checked by the oracle (-1: all), ncu summary in profiles/)
WORKLOADS = {
    'snowflake': ('config2', 2, 20_000_000, 10_000_000, 200_000, -1, 'root_scan_snowflake20M.md'),
    'tree': ('config3', 3, 10_000_000, 100_000, 20_000, 300, 'tree_level_10M.md'),
    'chowliu': ('config4', 4, 50_000_000, 20_000_000, 500_000, -1, 'pair_counts_chowliu50M.md'),
    'star': ('config1', 1, 200_000, 200_000, 200_000, -1, None),
}
# the sources a traffic figure in a profile depends on: the root scan's kernels
# (snowflake, Chow-Liu, star) or the tree pass's (tree)
TREE_SOURCES = ['paper_1906_08687_gb300/csrc/lmf_tree.cu',
                'paper_1906_08687_gb300/csrc/lmf_tree_dev.cuh',
                'paper_1906_08687_gb300/csrc/lmf_jit_tree.cu',
                'paper_1906_08687_gb300/csrc/lmf_rowpass.cuh',
                'paper_1906_08687_gb300/csrc/lmf_internal.h']
KERNEL_SOURCES = ['paper_1906_08687_gb300/csrc/lmf_kernels.cu',
                  'paper_1906_08687_gb300/csrc/lmf_gram_tc.cu',
                  'paper_1906_08687_gb300/csrc/lmf_rowpass.cuh',
                  'paper_1906_08687_gb300/csrc/lmf_root_plain.cuh',
                  'paper_1906_08687_gb300/csrc/lmf_root_lean.cuh',
                  'paper_1906_08687_gb300/csrc/lmf_root_tc.cuh',
                  'paper_1906_08687_gb300/csrc/lmf_jit.cu',
                  'paper_1906_08687_gb300/csrc/lmf_internal.h']


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=5)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--workload', default='snowflake', choices=sorted(WORKLOADS))
    ap.add_argument('--n-fact', type=int, default=None, help='fact rows (default: the workload\'s)')
    ap.add_argument('--precision', default='auto', choices=['auto', 'split', 'plain', 'plain-rowlevel'],
                    help='Gram form of the chosen plan; auto lets the learned plan choice '
                         '(shipped cost-model checkpoint, the Sec. 3.3 rule without one) pick the '
                         'root, the Gram form and view merging; split: split-bf16 tensor cores; '
                         'plain: FP32 (key-level blocks where eligible); plain-rowlevel: FP32, '
                         'every block per row')
    ap.add_argument('--fact-order', default='sorted', choices=['sorted', 'random'],
                    help='fact rows sorted by their join attributes (the input order of the '
                         "paper's experiments) or in generation order")
    ap.add_argument('--cpu-sample-rows', type=int, default=None)
    ap.add_argument('--ref-sample-rows', type=int, default=None)
    ap.add_argument('--check-aggs', type=int, default=None,
                    help='aggregates re-evaluated by the oracle over the full join (0: skip, -1: all)')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--shard', action='store_true',
                    help='one instance sharded over the ranks by root row ranges, partial results combined '
                         'by one all-reduce per result array (strong scaling); default: one instance per rank')
    args = ap.parse_args()
    gen, idx, n, cpu_rows, ref_rows, check, prof = WORKLOADS[args.workload]
    args.gen, args.cfg_index = gen, idx
    args.profile = os.path.join(ROOT, 'profiles', prof) if prof else ''
    args.n_fact = n if args.n_fact is None else args.n_fact
    args.cpu_sample_rows = cpu_rows if args.cpu_sample_rows is None else args.cpu_sample_rows
    args.ref_sample_rows = ref_rows if args.ref_sample_rows is None else args.ref_sample_rows
    args.check_aggs = check if args.check_aggs is None else args.check_aggs
    return args


def make_workload(args, rank=0):
    """The seeded schema and batch of the selected workload (rank r: seed + 1000 r)."""
    import workloads
    from workloads import SEED_BASE
    return getattr(workloads, args.gen)(args.n_fact, seed=SEED_BASE + args.cfg_index + 1000 * rank,
                                        fact_order=args.fact_order)


# ----------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = 'cuda' if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', f'--query-gpu={self.Q}', '--format=csv,noheader,nounits',
                                          '-i', str(self.index), '-lms', '200'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(',')]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == 'active':
                    reasons.add(n)
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': smax,
                'reasons': sorted(reasons), 'samples': len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {'hbm_gbs': d['hbm_gbs'], 'bf16_tflops': d['bf16_tflops'], 'source': 'measured'}
    return {'hbm_gbs': 6800.0, 'bf16_tflops': 1900.0, 'source': 'fallback'}


def kernel_hash(sources=None) -> str:
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(precision: str, summary: str, sources=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, when it was taken on the current kernel sources (else None)."""
    if not summary or not os.path.exists(summary):
        return None
    with open(summary) as f:
        text = f.read()
    m = re.search(rf'traffic_bytes_per_launch\[{precision}\]:\s*([0-9.e+]+)\s+sources:\s*([0-9a-f]+)', text)
    if not m or m.group(2) != kernel_hash(sources):
        return None
    return float(m.group(1))


def fact_order_text(sch, fact_order: str) -> str:
    """How the fact rows are ordered; a sorted root lists its join attributes in
    sort order (fewest distinct values first: the child with fewer keys)."""
    if fact_order != 'sorted':
        return 'generation order (i.i.d. rows)'
    keys = sorted((sch.rel(c).nrows, k) for p, c, k in sch.edges if p == sch.root)
    names = list(dict.fromkeys(k for _, k in keys))
    return (f"sorted by the join attributes, fewest distinct values first ({', '.join(names)}): "
            "the scan order of Sec. 3.5, as the paper's experiments load every relation")


WORKLOAD_TEXT = {
    'snowflake': '{name} (3 FKs, 8 fact + 22 dimension features, 10 categoricals; covar + grouped + pair counts)',
    'tree': '{name} (64 tree nodes x 20 features x <=32 thresholds x COUNT/SUM(y)/SUM(y^2))',
    'chowliu': '{name} (4 FKs, 30 categoricals; 435 pair counts, 30 marginals, 3-attribute cube)',
    'star': '{name} (2 FKs, 10 FP64 features; COUNT + all degree <= 2 monomials)',
}


# ----------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu's, else /proc/cpuinfo's, else the machine type)."""
    try:
        out = subprocess.run(['lscpu'], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith('Model name:'):
                return ln.split(':', 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open('/proc/cpuinfo') as f:
            for ln in f:
                if ln.lower().startswith('model name'):
                    return ln.split(':', 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_baseline(sch, batch, n_fact: int, sample_rows: int, single_thread: bool = False) -> dict:
    """The oracle, as it stands, on this host's cores over the first sample_rows
    fact rows of the workload (all aggregates); with single_thread also on one
    core."""
    from oracle import oracle
    oracle.build()
    S = min(sample_rows, n_fact)
    nt = oracle.max_threads()
    t0 = time.perf_counter()
    res = oracle.evaluate(sch, batch, root_range=(0, S), nthreads=nt)
    dt = time.perf_counter() - t0
    out = {'value': res.join_size * len(batch) / dt / 1e9, 'unit': UNIT, 'cores': nt,
           'kind': 'oracle', 'cpu': cpu_model(),
           'sample': f'first {S} fact rows of the same workload, all {len(batch)} aggregates ({dt:.1f} s)'}
    if single_thread:
        t0 = time.perf_counter()
        res1 = oracle.evaluate(sch, batch, root_range=(0, S), nthreads=1)
        dt1 = time.perf_counter() - t0
        out['value_1thread'] = res1.join_size * len(batch) / dt1 / 1e9
    return out


# ----------------------------------------------------------------------------
def run_reference(args):
    """The oracle on this host's cores, one bounded sample of the workload per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    oracle.build()
    sch, batch = make_workload(args)
    S = min(args.ref_sample_rows, args.n_fact)
    nt = oracle.max_threads()
    times = []
    for i in range(args.warmup + args.steps):
        b = (i * S) % max(1, args.n_fact - S + 1)
        t0 = time.perf_counter()
        res = oracle.evaluate(sch, batch, root_range=(b, b + S), nthreads=nt)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = res.join_size * len(batch) / t / 1e9
    sample = (f'{S} consecutive fact rows per step (of {args.n_fact}), all {len(batch)} aggregates, '
              f'full dimension tables')
    line = {
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': ws,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': t * 1e3, 'higher_is_better': True,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD_TEXT.get(args.workload, '{name}').format(name=sch.meta['name']),
                   'n_aggregates': len(batch),
                   'fact_order': fact_order_text(sch, args.fact_order),
                   'sample_rows_per_step': S},
        'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': nt, 'kind': 'oracle', 'cpu': cpu_model(),
                         'sample': sample},
        'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def run_sharded(args):
    """One instance of the workload sharded over the ranks: rank r registers the
    root rows row_range(N, r, world) with the dimensions whole, runs the batch
    and exports its packed results to device buffers, and one all-reduce (sum)
    per result array combines them (paper_1906_08687_gb300.shard).  A step is
    run + export + all-reduce; the step time is the maximum over ranks."""
    ws, rank, local = dist_env()
    import torch
    import torch.distributed as dist
    if ws > 1:
        dist.init_process_group('nccl')
    torch.cuda.set_device(local)
    from paper_1906_08687_gb300 import build as engine_build
    engine_build.build()
    from paper_1906_08687_gb300 import Engine, register_schema, shard
    from workloads import to_device
    sch, batch = make_workload(args, 0)            # the same instance on every rank
    n = sch.rel(sch.root).nrows
    b, e = shard.row_range(n, rank, ws)
    dev = to_device(sch, f'cuda:{local}')
    eng = Engine(local)
    register_schema(eng, shard.shard_schema(sch, b, e), shard.shard_tensors(sch, dev, b, e))
    bid = eng.declare_batch(batch)
    eng.plan(bid, precision=0, batching=1)
    info = eng.plan_info(bid)
    n_i, n_f = eng.result_sizes(bid)
    i64 = torch.zeros(max(1, n_i), dtype=torch.int64, device=f'cuda:{local}')
    f64 = torch.zeros(max(1, n_f), dtype=torch.float64, device=f'cuda:{local}')
    stream = torch.cuda.Stream()
    reduce = dist.all_reduce if ws > 1 else (lambda t: t)

    def step():
        eng.run(bid, stream.cuda_stream)
        eng.read_results(bid, i64.data_ptr(), f64.data_ptr(), True, stream.cuda_stream)
        with torch.cuda.stream(stream):
            shard.allreduce_packed(i64[:n_i], f64[:n_f], reduce)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ws, e0.elapsed_time(e1) / args.steps)
    eng.sync(bid)
    value = n * len(batch) / (ms * 1e-3) / 1e9
    line = {'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': ws, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': ms, 'higher_is_better': True, 'scaling': 'strong',
            'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
            'config': {'workload': WORKLOAD_TEXT.get(args.workload, '{name}').format(name=sch.meta['name']),
                       'n_aggregates': len(batch), 'join_rows': n, 'rows_per_rank': e - b,
                       'key_level': info['key_level'],
                       'parallelism': f'root row ranges x{ws}, one all-reduce per result array '
                                      f'({n_i} int64 + {n_f} float64 cells)'},
            'gpu_launches': info['n_kernels_per_run'] * args.steps}
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == 'reference':
        return run_reference(args)
    if args.shard:
        return run_sharded(args)
    ws, rank, local = dist_env()
    import numpy as np
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    torch.cuda.set_device(local)
    from paper_1906_08687_gb300 import build as engine_build
    engine_build.build()
    from paper_1906_08687_gb300 import Engine, register_schema
    from paper_1906_08687_gb300.lmf import STAGE_NAMES
    from workloads import to_device, to_pinned

    sch, batch = make_workload(args, rank)
    n_agg = len(batch)
    dev = to_device(sch, f'cuda:{local}')
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    def make(precision, batching, tensors, on_host=False, jit=True, opts=None):
        eng = Engine(local)
        register_schema(eng, sch, tensors, on_host=on_host)
        bid = eng.declare_batch(batch)
        if opts is not None:
            eng.plan_opts(bid, opts)
        else:
            eng.plan(bid, precision=precision, batching=batching, jit=jit)
        return eng, bid

    def timed(eng, bid, steps, warmup, sampler=None):
        for _ in range(warmup):
            eng.run(bid, sh)
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.start()
        e0.record(stream)
        for _ in range(steps):
            eng.run(bid, sh)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        barrier(ws)
        eng.sync(bid)
        return max_over_ranks(ws, e0.elapsed_time(e1) / steps), clocks

    # chosen form: the learned plan choice (lmf_plan_learned with the cost-model
    # checkpoint shipped in the package; the Sec. 3.3 root rule when there is
    # no usable checkpoint), one CUDA graph per run; --precision fixes the Gram
    # form instead
    from paper_1906_08687_gb300 import costmodel
    from paper_1906_08687_gb300.lmf import (LMF_BATCH_GRAPH, LMF_PLAN_ROW_GRAM, LMF_PREC_SPLIT_BF16,
                                            LMF_ROOT_HEURISTIC, lmf_plan_opts)
    base = lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, 0)
    names = {'split': 1, 'plain': 0}
    eng = Engine(local)
    register_schema(eng, sch, dev)
    bid = eng.declare_batch(batch)
    if args.precision == 'auto':
        model, origin = costmodel.load_shipped(local)
        chosen_opts = eng.plan_learned(bid, model, base)
    else:
        origin = f'fixed by --precision {args.precision}'
        prec_f = names[args.precision.split('-')[0]]
        flags = LMF_PLAN_ROW_GRAM if args.precision == 'plain-rowlevel' else 0
        eng.plan_opts(bid, lmf_plan_opts(prec_f, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, flags))
        chosen_opts = lmf_plan_opts(prec_f, LMF_BATCH_GRAPH, 0, 0, 1, eng.plan_info(bid)['root_rel'], 0, flags)
    # the rule's plan (Sec. 3.3 root, default options) for comparison
    e_r, b_r = make(None, None, dev, opts=lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0,
                                                        LMF_ROOT_HEURISTIC, 0, 0, 0))
    rule_ms, _ = timed(e_r, b_r, max(3, args.steps // 2), args.warmup)
    rule_info = e_r.plan_info(b_r)
    e_r.close()
    info = eng.plan_info(bid)
    prec = info['precision']
    join_rows = info['root_rows']   # unique dimension keys: |join| = fact rows
    sampler = ClockSampler(local)
    ms, clocks = timed(eng, bid, args.steps, args.warmup, sampler)
    value = ws * join_rows * n_agg / (ms * 1e-3) / 1e9

    info = eng.plan_info(bid)   # kernel count is known once the plan has run
    # per-stage device times (same plan, launched stage by stage with events)
    stage = np.zeros(len(STAGE_NAMES))
    for _ in range(args.steps):
        stage += np.array(eng.run_profiled(bid, sh))
    stage /= args.steps
    # the dominant stage: the root scan, or the tree pass for filtered batches
    dom_stage = max(('root_scan', 'tree'), key=lambda n: stage[STAGE_NAMES.index(n)])
    root_ms = float(stage[STAGE_NAMES.index(dom_stage)])

    # results of the chosen form for the accuracy check
    got = eng.results(bid, n_agg)

    # plain form: FP32 CUDA-core Gram, interpreted root scan (no plan-time
    # compile), kernels enqueued one by one
    eng_p, bid_p = make(0, 0, dev, jit=False)
    ms_plain, _ = timed(eng_p, bid_p, args.steps, args.warmup)
    eng_p.close()

    # end to end through the C ABI from pinned host buffers, every step moving
    # the step's inputs host -> device and reading the results back: the root's
    # columns read in place by the scan over the host link (LMF_HOST_MAPPED),
    # the dimensions copied; and everything copied (LMF_HOST_COPY)
    from paper_1906_08687_gb300.lmf import LMF_HOST_COPY, LMF_HOST_MAPPED
    host = to_pinned(sch)

    def e2e(modes):
        eng_e, bid_e = make(None, None, host, on_host=modes, opts=chosen_opts)
        n_i64, n_f64 = eng_e.result_sizes(bid_e)
        out_i = torch.empty(max(1, n_i64), dtype=torch.int64).pin_memory()
        out_f = torch.empty(max(1, n_f64), dtype=torch.float64).pin_memory()
        for _ in range(args.warmup):
            eng_e.run(bid_e, sh)
            eng_e.read_results(bid_e, out_i.data_ptr(), out_f.data_ptr(), False, sh)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            eng_e.run(bid_e, sh)
            eng_e.read_results(bid_e, out_i.data_ptr(), out_f.data_ptr(), False, sh)   # synchronous
        t = max_over_ranks(ws, (time.perf_counter() - t0) * 1e3 / args.steps)
        eng_e.sync(bid_e)
        eng_e.close()
        return t, 8 * (n_i64 + n_f64)

    e2e_ms, d2h = e2e({r.name: (LMF_HOST_MAPPED if r.name == sch.root else LMF_HOST_COPY)
                       for r in sch.relations})
    e2e_copy_ms, _ = e2e(LMF_HOST_COPY)
    h2d = sum(t.numel() * t.element_size() for t in host.values())

    # roofline of the root scan: algorithmic bytes = fact columns read once
    # plus every probed view record once
    R = sch.rel(sch.root)
    fact_bytes = sum(c.data.dtype.itemsize * R.nrows for c in R.columns)
    view_bytes = 0
    for r in sch.relations:
        if r.name != sch.root:
            view_bytes += sum(c.data.dtype.itemsize * r.nrows for c in r.columns)
    algo = fact_bytes + view_bytes
    peaks = measured_peaks()
    achieved = algo / (root_ms * 1e-3) / 1e9
    roof = {'bound': 'hbm', 'achieved': achieved, 'peak': peaks['hbm_gbs'], 'unit': 'GB/s',
            'frac': achieved / peaks['hbm_gbs'],
            'traffic': profiled_traffic('split' if prec == 1 else ('keylevel' if info['key_level'] else 'plain'),
                                        args.profile, TREE_SOURCES if dom_stage == 'tree' else KERNEL_SOURCES),
            'peak_source': peaks['source'], 'kernel': f'{dom_stage} stage',
            'algorithmic_bytes_per_launch': algo, 'launch_ms': root_ms,
            'stage_ms': {n: float(v) for n, v in zip(STAGE_NAMES, stage)}}

    line = {
        'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': ws, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': ms, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None,
        'dtype': 'bf16-split3/f32-acc' if info['precision'] == 1 else 'f32',
        'data': 'synthetic',
        'config': {'workload': WORKLOAD_TEXT.get(args.workload, '{name}').format(name=sch.meta['name']),
                   'n_aggregates': n_agg, 'join_rows': join_rows, 'precision': info['precision'],
                   'plan': {'origin': origin,
                            'root': sch.relations[info['root_rel']].name,
                            'gram': ('split-bf16 tcgen05' if prec == 1 else
                                     'FP32 root features + key-level blocks' if info['key_level'] else
                                     'FP32 CUDA cores, all blocks per row'),
                            'no_merge': int(chosen_opts.no_merge),
                            'root_scan_compiled': bool(info['jit']),
                            'resident_group': info['resident_group'],
                            'rule_plan': {'root': sch.relations[rule_info['root_rel']].name,
                                          'precision': rule_info['precision'],
                                          'key_level': rule_info['key_level'], 'ms_per_step': rule_ms}},
                   'fact_order': fact_order_text(sch, args.fact_order),
                   'batching': 'cuda-graph', 'kernels_per_step': info['n_kernels_per_run'],
                   'l2': f'inputs larger than L2 ({fact_bytes / 1e6:.0f} MB fact table per step)',
                   'parallelism': f'replicas x{ws}'},
        'hbm_pct_of_peak': 100.0 * roof['frac'],
        'speedup_vs_plain': ms_plain / ms, 'plain_ms_per_step': ms_plain,
        'plain_form': 'FP32 Gram, interpreted root scan, kernels launched one by one',
        'roofline': roof,
        'e2e': {'value': ws * join_rows * n_agg / (e2e_ms * 1e-3) / 1e9, 'unit': UNIT,
                'h2d_bytes_per_step': h2d, 'd2h_bytes_per_step': d2h, 'ms_per_step': e2e_ms,
                'inputs': 'pinned host memory; root columns read in place by the scan over the host '
                          'link (LMF_HOST_MAPPED), dimension columns copied by every run',
                'all_copied_ms_per_step': e2e_copy_ms},
        'gpu_launches': info['n_kernels_per_run'] * args.steps,
        'clocks': clocks,
    }

    if rank == 0 and args.check_aggs != 0:
        from oracle import oracle
        oracle.build()
        rng = np.random.default_rng(0)
        if args.check_aggs < 0 or args.check_aggs >= n_agg:
            pick = list(range(n_agg))
        else:
            pick = sorted(set([0] + list(rng.choice(n_agg, size=args.check_aggs, replace=False))))
        from oracle.compare import compare, compare_by_kind
        want = oracle.evaluate(sch, [batch[i] for i in pick])
        fails, stats = compare([got[i] for i in pick], want)
        line['accuracy'] = {'checked_aggregates': len(pick), 'failures': len(fails), **stats,
                            'rule': '|g-r| <= 1e-6*max(|r|, 1e-3*sum|v|); counts exact',
                            'by_kind': compare_by_kind([batch[i] for i in pick], [got[i] for i in pick], want)}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline(sch, batch, args.n_fact, args.cpu_sample_rows,
                                            single_thread=args.workload == 'star')
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == '__main__':
    sys.exit(main())
