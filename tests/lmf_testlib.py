"""Helpers shared by the GPU tests: upload a seeded schema, run it through the
C ABI, and compare with the oracle under the error rule of the tests.

Error rule (per aggregate cell): counts must be bit-exact; a sum g with oracle
value r and oracle scale A = SUM(|value|) must satisfy
    |g - r| <= 1e-6 * max(|r|, 1e-3 * A),
i.e. a relative error of 1e-6 wherever the sum is not a cancellation of
terms 1000x larger than itself.

Small inputs: the engine multiplies in 24-bit precision (FP32 products, or the
three-way bf16 split), so one product carries a relative error up to 2^-24
and a sum of products an error up to about 2^-24 * A.  With few rows the
rule above can be tighter than that (its floor 1e-9 * A only dominates the
statistical 2^-24 * sqrt(sum v^2) once the sum has ~10^4 terms), so tests on
small or ragged sizes also accept |g - r| <= ARITH_FLOOR * A.  Tests on the
benchmark configurations use the rule alone (arith_floor=0).
"""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-6
COND_FLOOR = 1e-3
ARITH_FLOOR = 2.0 ** -21


def to_device(schema, device='cuda:0'):
    import torch
    out = {}
    for r in schema.relations:
        for c in r.columns:
            out[(r.name, c.name)] = torch.from_numpy(np.ascontiguousarray(c.data)).to(device)
    return out


def to_pinned(schema):
    import torch
    out = {}
    for r in schema.relations:
        for c in r.columns:
            out[(r.name, c.name)] = torch.from_numpy(np.ascontiguousarray(c.data)).pin_memory()
    return out


def run_engine(schema, batch, precision=1, batching=1, tensors=None, runs=1, engine=None,
               tile_rows=0, ctas_per_sm=0, jit=True):
    """Register `schema`, declare and plan `batch`, run it `runs` times and
    return (list of per-aggregate numpy results of the last run, plan info)."""
    from paper_1906_08687_gb300 import Engine, register_schema
    eng = engine or Engine(0)
    tensors = tensors if tensors is not None else to_device(schema)
    register_schema(eng, schema, tensors)
    bid = eng.declare_batch(batch)
    eng.plan(bid, precision=precision, batching=batching, tile_rows=tile_rows,
             ctas_per_sm=ctas_per_sm, jit=jit)
    outs = []
    for _ in range(runs):
        eng.run(bid)
        eng.sync(bid)
        outs.append(eng.results(bid, len(batch)))
    info = eng.plan_info(bid)
    eng._tensors = tensors  # keep the borrowed buffers alive with the engine
    return (outs if runs > 1 else outs[0]), info, eng


def compare(got, want, arith_floor=0.0):
    """Return (failures, stats).  `want` is an oracle.OracleResult."""
    fails = []
    max_rel = 0.0
    max_ratio = 0.0
    for a, (g, r) in enumerate(zip(got, want.values)):
        g = np.asarray(g)
        if want.kinds[a] == 'count':
            if g.shape != r.shape or not np.array_equal(g.astype(np.int64), r):
                bad = np.nonzero(g != r)[0][:5] if g.shape == r.shape else 'shape'
                fails.append((a, 'count', bad))
            continue
        A = want.abs[a]
        err = np.abs(g - r)
        allow = np.maximum(REL_TOL * np.maximum(np.abs(r), COND_FLOOR * A), arith_floor * A)
        with np.errstate(divide='ignore', invalid='ignore'):
            rel = np.where(np.abs(r) > 0, err / np.abs(r), np.where(err > 0, np.inf, 0.0))
            ratio = np.where(allow > 0, err / allow, np.where(err > 0, np.inf, 0.0))
        if rel.size:
            max_rel = max(max_rel, float(np.max(rel[np.isfinite(rel)], initial=0.0)))
            max_ratio = max(max_ratio, float(np.max(ratio)))
        if np.any(err > allow):
            i = int(np.argmax(err - allow))
            fails.append((a, 'sum', dict(cell=i, got=float(g[i]), want=float(r[i]), A=float(A[i]))))
    return fails, {'max_raw_rel_err': max_rel, 'max_err_over_allowed': max_ratio}
