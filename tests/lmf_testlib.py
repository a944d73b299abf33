"""Helpers shared by the GPU tests: upload a seeded schema, run it through the
C ABI, and compare with the oracle under the error rule (oracle/compare.py:
counts bit-exact, sums |g - r| <= 1e-6 * max(|r|, 1e-3 * SUM(|value|)), with
an optional arithmetic floor for small or ragged inputs).
"""
from __future__ import annotations

from oracle.compare import ARITH_FLOOR, COND_FLOOR, REL_TOL, compare  # noqa: F401
from workloads import to_device, to_pinned  # noqa: F401


def run_engine(schema, batch, precision=1, batching=1, tensors=None, runs=1, engine=None,
               tile_rows=0, ctas_per_sm=0, jit=True, key_level=True):
    """Register `schema`, declare and plan `batch`, run it `runs` times and
    return (list of per-aggregate numpy results of the last run, plan info)."""
    from paper_1906_08687_gb300 import Engine, register_schema
    eng = engine or Engine(0)
    tensors = tensors if tensors is not None else to_device(schema)
    register_schema(eng, schema, tensors)
    bid = eng.declare_batch(batch)
    eng.plan(bid, precision=precision, batching=batching, tile_rows=tile_rows,
             ctas_per_sm=ctas_per_sm, jit=jit, key_level=key_level)
    outs = []
    for _ in range(runs):
        eng.run(bid)
        eng.sync(bid)
        outs.append(eng.results(bid, len(batch)))
    info = eng.plan_info(bid)
    eng._tensors = tensors  # keep the borrowed buffers alive with the engine
    return (outs if runs > 1 else outs[0]), info, eng
