"""Sharded evaluation of one batch over row ranges of the root relation.

The paper parallelises by partitioning the largest input relation (Sec. 1.2,
the parallelization layer).  Every aggregate of a batch is a sum over the
joined tuples (Eq. query), and the natural join partitions along the rows of
the root: every joined tuple extends exactly one root row.  So rank r
registers the rows row_range(N, r, world) of the root, with every other
relation whole (the views are small and built on every rank), evaluates the
whole batch over its rows, and one all-reduce (sum) of the two result arrays
-- exact int64 counts and FP64 sums, packed in the engine's result layout --
gives the batch over the whole join.  Integer sums are exact in any order; the
FP64 sums of the ranks' partials differ from a single run only by rounding
order (~1e-16 relative).

Marshalling and host logic only: every aggregate is computed by the engine's
kernels on each rank; the exchange is torch.distributed's all_reduce (NCCL on
GPUs, gloo on CPU).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Sequence, Tuple

import numpy as np


def row_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Rows [begin, end) of the root that rank `rank` of `world` evaluates:
    contiguous, in rank order, sizes differing by at most one, together every
    row exactly once."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError(f'rank {rank} of {world}')
    return n * rank // world, n * (rank + 1) // world


def shard_schema(schema, begin: int, end: int):
    """The schema with its root cut to rows [begin, end) (numpy views, no copy)."""
    root = schema.rel(schema.root)
    part = type(root)(root.name, [dataclasses.replace(c, data=c.data[begin:end]) for c in root.columns])
    rels = [part if r.name == schema.root else r for r in schema.relations]
    return type(schema)(rels, schema.edges, schema.root, dict(schema.meta))


def shard_tensors(schema, tensors: dict, begin: int, end: int) -> dict:
    """Column buffers of the shard: the root's columns sliced to [begin, end)
    (views of the same memory, so their data pointers are offset), the rest
    as given."""
    out = dict(tensors)
    for c in schema.rel(schema.root).columns:
        out[(schema.root, c.name)] = tensors[(schema.root, c.name)][begin:end]
    return out


def result_layout(schema, batch: Sequence) -> Tuple[List[Tuple[bool, int, int]], int, int]:
    """The engine's packed result layout of a batch: per aggregate (is_count,
    cells, offset) -- counts (no power factor) in the int64 array, sums in the
    float64 array, each in aggregate order, cells the product of the group-by
    domains -- and the two array lengths (lmf_result_info, lmf_result_sizes)."""
    dom = {}
    for r in schema.relations:
        for c in r.columns:
            if c.role == 'cat':
                dom[c.name] = int(c.cat_domain)
    out, n_i, n_f = [], 0, 0
    for a in batch:
        cells = 1
        for g in a.group_by:
            cells *= dom[g]
        is_count = not any(f[1] == 'pow' for f in a.factors)
        if is_count:
            out.append((True, cells, n_i))
            n_i += cells
        else:
            out.append((False, cells, n_f))
            n_f += cells
    return out, n_i, n_f


def pack(results: Sequence[np.ndarray], schema, batch) -> Tuple[np.ndarray, np.ndarray]:
    """Per-aggregate result arrays -> the packed (int64, float64) arrays."""
    layout, n_i, n_f = result_layout(schema, batch)
    i64 = np.zeros(n_i, np.int64)
    f64 = np.zeros(n_f, np.float64)
    for (is_count, n, off), r in zip(layout, results):
        r = np.asarray(r).reshape(-1)
        if r.size != n:
            raise ValueError(f'aggregate has {r.size} cells, the layout {n}')
        if is_count:
            i64[off:off + n] = r
        else:
            f64[off:off + n] = r
    return i64, f64


def unpack(i64: np.ndarray, f64: np.ndarray, schema, batch) -> List[np.ndarray]:
    """The packed arrays -> one array per aggregate (copies)."""
    layout, _, _ = result_layout(schema, batch)
    return [(i64 if is_count else f64)[off:off + n].copy() for is_count, n, off in layout]


def allreduce_packed(i64, f64, all_reduce: Callable) -> None:
    """Sum the packed arrays of every rank in place: one all-reduce per array
    (torch tensors; all_reduce is torch.distributed.all_reduce or a stand-in).
    Empty arrays are skipped."""
    for t in (i64, f64):
        if t.numel() > 0:
            all_reduce(t)
